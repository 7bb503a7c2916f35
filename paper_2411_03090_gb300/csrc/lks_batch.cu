// lks_batch.cu -- the batched form of the C ABI (lks_batch_* in include/lks.h): many
// unsteady designs of unequal lattice size marched in lock step, one persistent
// launch per time step over a work list of (design, tile) pairs, the whole gradient
// captured as one CUDA graph, and a tile shape picked by timing.
//
// Per design the computation is that of lks_forward + alks_adjoint +
// lks_sensitivity for an unsteady FP32 problem with checkpoints every K steps
// (arXiv 2411.03090, Sec. 2.7 Steps 2-5): the forward march stores a snapshot of
// (drho, u, v) every K steps; the adjoint re-runs each segment forward from its
// snapshot, keeping the segment's (u, v) levels, and marches the ALKS backward over
// it while accumulating the sensitivity (FP32, flushed to FP64 every 256 levels).
// The step kernels are the TMA kernels of lks_tma.cuh instantiated with BATCH =
// true, so each node sees the arithmetic of the single-lattice form.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/lks.h"
#include "lks_host.cuh"
#include "lks_kernels.cuh"
#include "lks_col.cuh"
#include "lks_tma.cuh"

using namespace lks;
using namespace lks_host;

namespace {

constexpr int kNCfg = LKS_BATCH_TILE_CONFIGS;
constexpr int kAlignX = 128, kAlignY = 16;  // rectangle granularity: every tile shape divides it
constexpr int kFwdNTb = 256, kAdjNTb = 512;
constexpr int kJBX = 32;   // objective blocks per design
constexpr int kEwBX = 32;  // blocks per design of the per-design elementwise kernels
constexpr int kFlushEvery = 256;

struct TileShape {
  int tx, ty;
};
constexpr TileShape kShape[kNCfg] = {{64, 8}, {32, 16}, {128, 4}, {64, 16}};

inline size_t up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ------------------------------------------------------------------------------------
// Batch kernels (per design rectangle: blockIdx.y = design)
// ------------------------------------------------------------------------------------
__global__ void scatter_gamma_kernel(const float* const* __restrict__ src, float* __restrict__ arena,
                                     const BatchDesign* __restrict__ dz, int pitch) {
  const BatchDesign& bd = dz[blockIdx.y];
  const float* s = src[blockIdx.y];
  const int nx = bd.g.nx;
  const size_t n = (size_t)nx * bd.g.ny;
  for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(o / nx), i = (int)(o - (size_t)j * nx);
    arena[(size_t)(bd.ay + j) * pitch + bd.ax + i] = s[o];
  }
}

__global__ void fill_gamma_kernel(float value, float* __restrict__ arena, const BatchDesign* __restrict__ dz,
                                  int pitch) {
  const BatchDesign& bd = dz[blockIdx.y];
  const int nx = bd.g.nx;
  const size_t n = (size_t)nx * bd.g.ny;
  for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(o / nx), i = (int)(o - (size_t)j * nx);
    arena[(size_t)(bd.ay + j) * pitch + bd.ax + i] = value;
  }
}

// 1 / (1 + alpha_gamma) and alpha_gamma (Eq. brinkman) with each design's alpha_bar, q.
__global__ void batch_material_kernel(const float* __restrict__ gamma, const BatchDesign* __restrict__ dz, int pitch,
                                      float* __restrict__ binv, float* __restrict__ alpha) {
  const BatchDesign& bd = dz[blockIdx.y];
  const int nx = bd.g.nx;
  const size_t n = (size_t)nx * bd.g.ny;
  for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(o / nx), i = (int)(o - (size_t)j * nx);
    const size_t p = (size_t)(bd.ay + j) * pitch + bd.ax + i;
    const float al = alpha_of(bd.c, gamma[p]);
    binv[p] = 1.f / (1.f + al);
    alpha[p] = al;
  }
}

// J_O of each design's state (total dissipation, interior nodes): partial[d][block].
template <int NT>
__global__ void __launch_bounds__(NT) batch_objective_kernel(const float* __restrict__ u, const float* __restrict__ v,
                                                             const float* __restrict__ gamma,
                                                             const BatchDesign* __restrict__ dz, int pitch,
                                                             double* __restrict__ partial) {
  __shared__ double red[NT / 32];
  const BatchDesign& bd = dz[blockIdx.y];
  const int nx = bd.g.nx, ny = bd.g.ny;
  const Coef<float>& c = bd.c;
  const size_t n = (size_t)nx * ny;
  double acc = 0.0;
  for (size_t o = (size_t)blockIdx.x * NT + threadIdx.x; o < n; o += (size_t)gridDim.x * NT) {
    const int j = (int)(o / nx), i = (int)(o - (size_t)j * nx);
    if (i == 0 || j == 0 || i == nx - 1 || j == ny - 1) continue;
    const size_t p = (size_t)(bd.ay + j) * pitch + bd.ax + i;
    const float dudx = (u[p + 1] - u[p - 1]) * 0.5f, dudy = (u[p + pitch] - u[p - pitch]) * 0.5f;
    const float dvdx = (v[p + 1] - v[p - 1]) * 0.5f, dvdy = (v[p + pitch] - v[p - pitch]) * 0.5f;
    const float Sxx = 2.f * dudx, Syy = 2.f * dvdy, Sxy = dudy + dvdx;
    const float al = alpha_of(c, gamma[p]);
    acc += (double)(0.5f * c.nu * (Sxx * Sxx + 2.f * Sxy * Sxy + Syy * Syy) + al * (u[p] * u[p] + v[p] * v[p]));
  }
  const double s = block_sum<NT>(acc, red);
  if (threadIdx.x == 0) partial[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
}

// J of design d: its per-tile step partials (tiles rng[2d] .. rng[2d+1]) plus the
// final-state partials, summed in a fixed order.
__global__ void batch_reduce_J_kernel(const double* __restrict__ jt, const int* __restrict__ rng,
                                      const double* __restrict__ jfin, int jbx, double* __restrict__ out) {
  __shared__ double red[NTHREADS / 32];
  const int d = blockIdx.x;
  double acc = 0.0;
  for (int q = rng[2 * d] + threadIdx.x; q < rng[2 * d + 1]; q += NTHREADS) acc += jt[q];
  for (int q = threadIdx.x; q < jbx; q += NTHREADS) acc += jfin[(size_t)d * jbx + q];
  const double s = block_sum<NTHREADS>(acc, red);
  if (threadIdx.x == 0) out[d] = s;
}

__global__ void gather_grad_kernel(const double* __restrict__ sens64, float* const* __restrict__ dst,
                                   const BatchDesign* __restrict__ dz, int pitch) {
  const BatchDesign& bd = dz[blockIdx.y];
  float* y = dst[blockIdx.y];
  const int nx = bd.g.nx;
  const size_t n = (size_t)nx * bd.g.ny;
  for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(o / nx), i = (int)(o - (size_t)j * nx);
    y[o] = (float)(sens64[(size_t)(bd.ay + j) * pitch + bd.ax + i] + 0.0);
  }
}

// Snapshot codec with one max-abs scale per design and field.
__global__ void batch_absmax_kernel(const float* __restrict__ x, const BatchDesign* __restrict__ dz, int pitch,
                                    float* __restrict__ scale) {
  const BatchDesign& bd = dz[blockIdx.y];
  const int nx = bd.g.nx;
  const size_t n = (size_t)nx * bd.g.ny;
  float m = 0.f;
  for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(o / nx), i = (int)(o - (size_t)j * nx);
    m = fmaxf(m, fabsf(x[(size_t)(bd.ay + j) * pitch + bd.ax + i]));
  }
  for (int s = 16; s > 0; s >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, s));
  if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int*>(scale + blockIdx.y), __float_as_int(m));
}

template <typename S>
__device__ __forceinline__ S enc_val(float v);
template <>
__device__ __forceinline__ __nv_bfloat16 enc_val<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}
template <>
__device__ __forceinline__ __half enc_val<__half>(float v) {
  return __float2half_rn(v);
}
__device__ __forceinline__ float dec_val(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float dec_val(__half v) { return __half2float(v); }

template <typename S>
__global__ void batch_encode_kernel(const float* __restrict__ x, S* __restrict__ y, const BatchDesign* __restrict__ dz,
                                    int pitch, const float* __restrict__ scale) {
  const BatchDesign& bd = dz[blockIdx.y];
  const float s = scale[blockIdx.y];
  const float inv = s > 0.f ? 1.f / s : 0.f;
  const int nx = bd.g.nx;
  const size_t n = (size_t)nx * bd.g.ny;
  for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(o / nx), i = (int)(o - (size_t)j * nx);
    const size_t p = (size_t)(bd.ay + j) * pitch + bd.ax + i;
    y[p] = enc_val<S>(x[p] * inv);
  }
}
template <typename S>
__global__ void batch_decode_kernel(const S* __restrict__ y, float* __restrict__ x, const BatchDesign* __restrict__ dz,
                                    int pitch, const float* __restrict__ scale) {
  const BatchDesign& bd = dz[blockIdx.y];
  const float s = scale[blockIdx.y];
  const int nx = bd.g.nx;
  const size_t n = (size_t)nx * bd.g.ny;
  for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(o / nx), i = (int)(o - (size_t)j * nx);
    const size_t p = (size_t)(bd.ay + j) * pitch + bd.ax + i;
    x[p] = dec_val(y[p]) * s;
  }
}

// ------------------------------------------------------------------------------------
// Plan: arena packing, work lists, checkpoint spacing and workspace layout
// ------------------------------------------------------------------------------------
// Work lists 0 .. kNCfg-1 belong to the tile shapes of the TMA-staged kernels, list
// kColList to the warp-column forward (60 x 40 tiles), kAdjColList to the
// warp-column adjoint (28 x 32 tiles).
constexpr int kColList = kNCfg;
constexpr int kAdjColList = kNCfg + 1;
constexpr int kNLists = kNCfg + 2;
struct BLayout {
  size_t designs = 0, work[kNLists] = {}, rng[kNLists] = {}, uin = 0, emap = 0, gptr = 0, dptr = 0;
  size_t gamma = 0, stA = 0, stB = 0, adA = 0, adB = 0, mat = 0, sens = 0, sens64 = 0;
  size_t jt = 0, jfin = 0, jval = 0, status = 0, snaps = 0, scales = 0, seg = 0, seg2 = 0, total = 0;
};

struct Plan {
  int n = 0, W = 0, H = 0, n_steps = 0, K = 0, n_ckpt = 0, seg_levels = 0, snap_type = LKS_SNAP_BF16;
  size_t A = 0, snap_elem = 2;
  int64_t nodes = 0;
  std::vector<int> ax, ay;
  std::vector<BatchTile> work[kNLists];
  std::vector<int> rng[kNLists];
  BLayout L;
};

// Shelf packing of rectangles (fw, fh) into width W: tallest first, left to right.
int shelf_pack(const std::vector<int>& fw, const std::vector<int>& fh, int W, std::vector<int>& ax,
               std::vector<int>& ay) {
  const int n = (int)fw.size();
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return fh[a] > fh[b]; });
  int x = 0, y = 0, sh = 0;
  for (int d : order) {
    if (x + fw[d] > W) {
      y += sh;
      x = 0;
      sh = 0;
    }
    ax[d] = x;
    ay[d] = y;
    x += fw[d];
    sh = std::max(sh, fh[d]);
  }
  return y + sh;
}

// Checkpoint spacing that minimises snapshot + segment-store bytes (two segment
// stores: the recompute of a segment overlaps the adjoint of the next).
int memory_optimal_K(int n_steps, size_t A, size_t se) {
  size_t best = SIZE_MAX;
  int bk = 1;
  for (int K = 1; K <= n_steps; ++K) {
    const size_t nck = (size_t)((n_steps + K - 1) / K);
    const size_t bytes = nck * 3 * A * se + 2 * (size_t)(K + 2) * 2 * A * 4;
    if (bytes < best) {
      best = bytes;
      bk = K;
    }
  }
  return bk;
}

lks_batch_options default_options() {
  lks_batch_options o;
  std::memset(&o, 0, sizeof(o));
  o.version = LKS_BATCH_VERSION;
  o.checkpoint_every = 0;
  o.snapshot_type = LKS_SNAP_BF16;
  o.tile_config = -1;
  o.use_graph = 1;
  o.fwd_column = -1;
  o.adj_column = -1;
  return o;
}

lks_status make_plan(int32_t n, const lks_problem_desc* descs, const lks_batch_options* opt, Plan* P,
                     std::string* why) {
  auto bad = [&](const std::string& m) {
    if (why) *why = m;
    return LKS_ERR_INVALID_ARG;
  };
  if (n < 1 || n > 65535) return bad("n_designs must lie in [1, 65535]");
  if (!descs) return bad("descs is NULL");
  if (opt->version != LKS_BATCH_VERSION) return bad("batch options version mismatch");
  if (opt->checkpoint_every < 0) return bad("checkpoint_every must be >= 0");
  if (opt->snapshot_type < LKS_SNAP_F32 || opt->snapshot_type > LKS_SNAP_F16) return bad("bad snapshot_type");
  if (opt->tile_config < -1 || opt->tile_config >= kNCfg) return bad("bad tile_config");
  if (opt->use_graph != 0 && opt->use_graph != 1) return bad("use_graph must be 0 or 1");
  if (opt->fwd_column < -1 || opt->fwd_column > 1) return bad("fwd_column must be -1, 0 or 1");
  if (opt->adj_column < -1 || opt->adj_column > 1) return bad("adj_column must be -1, 0 or 1");
  for (int q = 0; q < 5; ++q)
    if (opt->reserved[q] != 0) return bad("reserved option fields must be zero");
  P->n = n;
  P->n_steps = descs[0].n_steps;
  std::vector<int> fw(n), fh(n);
  int maxw = 0;
  for (int d = 0; d < n; ++d) {
    std::string w;
    if (check_desc(&descs[d], &w) != LKS_OK) return bad("design " + std::to_string(d) + ": " + w);
    if (descs[d].real_type != LKS_REAL_F32) return bad("batched designs must be FP32");
    if (descs[d].steady) return bad("batched designs must be unsteady");
    if (descs[d].thermal) return bad("batched designs must be non-thermal");
    if (descs[d].kappa_E != 0.0) return bad("batched designs: kappa_E must be 0");
    if (descs[d].lattice != LKS_LATTICE_D2Q9) return bad("batched designs must be D2Q9");
    if (descs[d].n_steps != P->n_steps) return bad("batched designs must share n_steps");
    fw[d] = (int)up(descs[d].nx, kAlignX);
    fh[d] = (int)up(descs[d].ny, kAlignY);
    maxw = std::max(maxw, fw[d]);
    P->nodes += (int64_t)descs[d].nx * descs[d].ny;
  }
  // arena width: the multiple of 128 (up to 16384) whose shelf packing has least area
  P->ax.assign(n, 0);
  P->ay.assign(n, 0);
  size_t best = SIZE_MAX;
  int bestW = maxw;
  std::vector<int> tx(n), ty(n);
  for (int W = maxw; W <= std::max(maxw, 16384); W += kAlignX) {
    const int H = shelf_pack(fw, fh, W, tx, ty);
    const size_t area = (size_t)W * H;
    if (area < best) {
      best = area;
      bestW = W;
    }
  }
  P->W = bestW;
  P->H = shelf_pack(fw, fh, bestW, P->ax, P->ay);
  P->A = (size_t)P->W * P->H;
  if (P->A > ((size_t)1 << 31)) return bad("arena larger than 2^31 nodes");
  // work lists, design by design, row-major tiles
  for (int c = 0; c < kNLists; ++c) {
    const int TXc = c < kNCfg ? kShape[c].tx : c == kColList ? C2_W : COL_W;
    const int TYc = c < kNCfg ? kShape[c].ty : c == kColList ? Col2Geo<C2_R>::H : ACOL_H;
    P->work[c].clear();
    P->rng[c].assign(2 * n, 0);
    for (int d = 0; d < n; ++d) {
      const int nx = descs[d].nx, ny = descs[d].ny;
      P->rng[c][2 * d] = (int)P->work[c].size();
      for (int y0 = 0; y0 < ny; y0 += TYc)
        for (int x0 = 0; x0 < nx; x0 += TXc) {
          BatchTile t;
          t.d = d;
          t.x0 = x0;
          t.y0 = y0;
          t.interior = (x0 >= 2 && y0 >= 2 && x0 + TXc + 2 <= nx && y0 + TYc + 2 <= ny) ? 1 : 0;
          P->work[c].push_back(t);
        }
      P->rng[c][2 * d + 1] = (int)P->work[c].size();
    }
  }
  P->snap_type = opt->snapshot_type;
  P->snap_elem = opt->snapshot_type == LKS_SNAP_F32 ? 4 : 2;
  P->K = opt->checkpoint_every > 0 ? std::min(opt->checkpoint_every, P->n_steps)
                                   : memory_optimal_K(P->n_steps, P->A, P->snap_elem);
  P->n_ckpt = (P->n_steps + P->K - 1) / P->K;
  P->seg_levels = P->K + 2;
  // layout
  BLayout& L = P->L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = up(off + bytes, 256);
    return o;
  };
  size_t max_tiles = 0;
  L.designs = take(sizeof(BatchDesign) * n);
  for (int c = 0; c < kNLists; ++c) {
    L.work[c] = take(sizeof(BatchTile) * P->work[c].size());
    L.rng[c] = take(sizeof(int) * 2 * n);
    max_tiles = std::max(max_tiles, P->work[c].size());
  }
  L.uin = take(sizeof(float) * (size_t)n * (P->n_steps + 1));
  L.emap = take(sizeof(float) * (size_t)n * 540);
  L.gptr = take(sizeof(void*) * n);
  L.dptr = take(sizeof(void*) * n);
  const size_t fb = P->A * 4;
  L.gamma = take(fb);
  L.stA = take(fb * 3);
  L.stB = take(fb * 3);
  L.adA = take(fb * 6);
  L.adB = take(fb * 6);
  L.mat = take(fb * 2);
  L.sens = take(fb);
  L.sens64 = take(P->A * 8);
  L.jt = take(sizeof(double) * max_tiles);
  L.jfin = take(sizeof(double) * (size_t)n * kJBX);
  L.jval = take(sizeof(double) * n);
  L.status = take(sizeof(int));
  L.snaps = take(P->snap_elem * P->A * 3 * (size_t)P->n_ckpt);
  L.scales = take(sizeof(float) * 3 * (size_t)n * P->n_ckpt);
  L.seg = take(fb * 2 * (size_t)P->seg_levels);
  L.seg2 = take(fb * 2 * (size_t)P->seg_levels);
  L.total = off;
  return LKS_OK;
}

}  // namespace

// ------------------------------------------------------------------------------------
// Handle
// ------------------------------------------------------------------------------------
struct lks_batch {
  int n = 0;
  std::vector<lks_problem_desc> d;
  lks_batch_options opt;
  Plan P;
  unsigned char* ws = nullptr;
  size_t ws_bytes = 0;
  cudaStream_t stream = nullptr;
  int device = 0, sms = 0;
  int cfg = 0;
  bool fwd_col = false;  // forward on the warp-column kernel (work list kColList)
  bool adj_col = false;  // adjoint on the warp-column kernel (work list kAdjColList)
  int grid_fwd[kNCfg] = {}, grid_adj[kNCfg] = {};
  int cur = 0, acur = 0;
  std::unordered_map<uint64_t, CUtensorMap> tmaps;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t launches = 0, launches_per_grad = 0, gradients = 0;
  float tune_us[kNCfg] = {}, tune_fwd_us[kNCfg] = {}, tune_col_us = 0.f, tune_acol_us = 0.f;
  std::string err;
  // The segment recompute runs on a second stream, overlapped with the adjoint of
  // the next segment (a parallel branch of the captured graph); events order the
  // two segment stores between the streams.
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_seg[2] = {nullptr, nullptr}, ev_adj[2] = {nullptr, nullptr};
  ~lks_batch() {
    for (cudaEvent_t e : {ev_fork, ev_seg[0], ev_seg[1], ev_adj[0], ev_adj[1]})
      if (e) cudaEventDestroy(e);
    if (aux) cudaStreamDestroy(aux);
  }
};

namespace {

lks_status bfail(lks_batch* b, lks_status s, const std::string& m) {
  if (b) b->err = m;
  return s;
}

#define CKB(b, call)                                                                     \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return bfail(b, LKS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

float* af(lks_batch* b, size_t off, int k = 0) { return reinterpret_cast<float*>(b->ws + off) + (size_t)k * b->P.A; }
float* stp(lks_batch* b, int which, int f) { return af(b, which == 0 ? b->P.L.stA : b->P.L.stB, f); }
float* adp(lks_batch* b, int which, int f) { return af(b, which == 0 ? b->P.L.adA : b->P.L.adB, f); }
const BatchDesign* ddesigns(lks_batch* b) { return reinterpret_cast<const BatchDesign*>(b->ws + b->P.L.designs); }
int* dstatus(lks_batch* b) { return reinterpret_cast<int*>(b->ws + b->P.L.status); }

// Tensor map of one arena field (W x H floats) for boxes bw x bh, cached.
lks_status arena_map(lks_batch* b, const void* ptr, int bw, int bh, CUtensorMap* out) {
  const uint64_t key = reinterpret_cast<uint64_t>(ptr) ^ ((uint64_t)bw << 48) ^ ((uint64_t)bh << 56);
  auto it = b->tmaps.find(key);
  if (it != b->tmaps.end()) {
    *out = it->second;
    return LKS_OK;
  }
  CUtensorMap m;
  const cuuint64_t dims[2] = {(cuuint64_t)b->P.W, (cuuint64_t)b->P.H};
  const cuuint64_t strides[1] = {(cuuint64_t)b->P.W * 4};
  const cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(ptr), dims, strides, box, es,
                                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return bfail(b, LKS_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  b->tmaps.emplace(key, m);
  *out = m;
  return LKS_OK;
}

template <int C>
constexpr size_t fwd_smem() {
  return fwd_tma_smem_bytes<false, kShape[C].tx, kShape[C].ty>();
}
template <int C>
constexpr size_t adj_smem() {
  return adj_tma_smem_bytes<false, false, kShape[C].tx, kShape[C].ty>();
}

template <int C>
lks_status setup_cfg(lks_batch* b) {
  constexpr int TXc = kShape[C].tx, TYc = kShape[C].ty;
  auto fk = fwd_tma_kernel<false, true, TXc, TYc, kFwdNTb>;
  auto ak = adj_tma_kernel<false, false, true, TXc, TYc, kAdjNTb>;
  CKB(b, cudaFuncSetAttribute(fk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem<C>()));
  CKB(b, cudaFuncSetAttribute(ak, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)adj_smem<C>()));
  int pf = 0, pa = 0;
  CKB(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pf, fk, kFwdNTb, fwd_smem<C>()));
  CKB(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pa, ak, kAdjNTb, adj_smem<C>()));
  const int nt = (int)b->P.work[C].size();
  b->grid_fwd[C] = std::max(1, std::min(nt, std::max(pf, 1) * b->sms));
  b->grid_adj[C] = std::max(1, std::min(nt, std::max(pa, 1) * b->sms));
  return LKS_OK;
}

// One forward step of every design: state cur -> other buffer, level t_new.
template <int C>
lks_status fwd_step_c(lks_batch* b, int t_new, bool jacc, float* tu, float* tv) {
  constexpr int TXc = kShape[C].tx, TYc = kShape[C].ty;
  const int src = b->cur, dst = 1 - b->cur;
  TmaMaps<4> maps;
  lks_status st;
  const float* fsrc[4] = {stp(b, src, 0), stp(b, src, 1), stp(b, src, 2), af(b, b->P.L.mat, 0)};
  for (int f = 0; f < 4; ++f)
    if ((st = arena_map(b, fsrc[f], TXc + 8, TYc + 4, &maps.m[f])) != LKS_OK) return st;
  FwdOutMaps<false> omaps;
  const float* outs[5] = {stp(b, dst, 0), stp(b, dst, 1), stp(b, dst, 2), tu, tv};
  for (int f = 0; f < 5; ++f)
    if (outs[f] && (st = arena_map(b, outs[f], TXc, TYc, &omaps.m[f])) != LKS_OK) return st;
  FwdTmaArgs<false> a;
  std::memset(&a, 0, sizeof(a));
  a.drho_n = stp(b, dst, 0);
  a.u_n = stp(b, dst, 1);
  a.v_n = stp(b, dst, 2);
  a.gamma = af(b, b->P.L.gamma);
  a.J_partial = jacc ? reinterpret_cast<double*>(b->ws + b->P.L.jt) : nullptr;
  a.status = dstatus(b);
  a.traj_u = tu;
  a.traj_v = tv;
  a.ntiles = (int)b->P.work[C].size();
  a.work = reinterpret_cast<const BatchTile*>(b->ws + b->P.L.work[C]);
  a.designs = ddesigns(b);
  a.u_in_d = reinterpret_cast<const float*>(b->ws + b->P.L.uin) + (size_t)t_new * b->n;
  fwd_tma_kernel<false, true, TXc, TYc, kFwdNTb>
      <<<b->grid_fwd[C], kFwdNTb, fwd_smem<C>(), b->stream>>>(maps, omaps, a, Geom{}, Coef<float>{});
  CKB(b, cudaGetLastError());
  b->cur = dst;
  b->launches++;
  return LKS_OK;
}

// One adjoint step of every design: adjoint acur -> other buffer with the state
// levels (u1, v1) at t+1 and (u0, v0) at t; sensitivity accumulated when sens_flow.
template <int C>
lks_status adj_step_c(lks_batch* b, const float* u1, const float* v1, const float* u0, const float* v0,
                      int sens_flow) {
  constexpr int TXc = kShape[C].tx, TYc = kShape[C].ty;
  constexpr int NF = adj_tma_nf(false, false);
  const int src = b->acur, dst = 1 - b->acur;
  TmaMaps<NF> maps;
  lks_status st;
  const float* mat = af(b, b->P.L.mat, 0);
  const float* fsrc[NF] = {adp(b, src, 0), adp(b, src, 1), adp(b, src, 2), adp(b, src, 3), adp(b, src, 4),
                           adp(b, src, 5), u1, v1, u0, v0, mat + b->P.A, mat};  // ..., alpha, 1/(1+alpha)
  for (int f = 0; f < NF; ++f)
    if ((st = arena_map(b, fsrc[f], TXc + 8, TYc + 4, &maps.m[f])) != LKS_OK) return st;
  AdjOutMaps<false> omaps;
  for (int f = 0; f < 6; ++f)
    if ((st = arena_map(b, adp(b, dst, f), TXc, TYc, &omaps.m[f])) != LKS_OK) return st;
  AdjTmaArgs<false> a;
  std::memset(&a, 0, sizeof(a));
  for (int q = 0; q < 9; ++q) a.m0[q] = adp(b, dst, q < 6 ? q : 0);
  a.gamma = af(b, b->P.L.gamma);
  a.emap = reinterpret_cast<const float*>(b->ws + b->P.L.emap);
  a.sens = af(b, b->P.L.sens);
  a.sens_flow = sens_flow;
  a.sens_thermal = 0;
  a.status = dstatus(b);
  a.ntiles = (int)b->P.work[C].size();
  a.work = reinterpret_cast<const BatchTile*>(b->ws + b->P.L.work[C]);
  a.designs = ddesigns(b);
  a.pitch = b->P.W;
  adj_tma_kernel<false, false, true, TXc, TYc, kAdjNTb>
      <<<b->grid_adj[C], kAdjNTb, adj_smem<C>(), b->stream>>>(maps, omaps, a, Geom{}, Coef<float>{});
  CKB(b, cudaGetLastError());
  b->acur = dst;
  b->launches++;
  return LKS_OK;
}

// One forward step of every design on the warp-column kernel (one CTA per entry of
// work list kColList).
lks_status fwd_col_step(lks_batch* b, int t_new, bool jacc, float* tu, float* tv) {
  using G2 = Col2Geo<C2_R>;
  const int src = b->cur, dst = 1 - b->cur;
  TmaMaps<4> maps;
  lks_status st;
  const float* fsrc[4] = {stp(b, src, 0), stp(b, src, 1), stp(b, src, 2), af(b, b->P.L.mat, 0)};
  for (int f = 0; f < 4; ++f)
    if ((st = arena_map(b, fsrc[f], C2_BW, G2::BH, &maps.m[f])) != LKS_OK) return st;
  Col2Args a;
  std::memset(&a, 0, sizeof(a));
  for (int f = 0; f < 3; ++f) a.out[f] = stp(b, dst, f);
  a.traj_u = tu;
  a.traj_v = tv;
  a.J_partial = jacc ? reinterpret_cast<double*>(b->ws + b->P.L.jt) : nullptr;
  a.status = dstatus(b);
  a.work = reinterpret_cast<const BatchTile*>(b->ws + b->P.L.work[kColList]);
  a.designs = ddesigns(b);
  a.u_in_d = reinterpret_cast<const float*>(b->ws + b->P.L.uin) + (size_t)t_new * b->n;
  a.pitch = b->P.W;
  fwd_col2_kernel<C2_R, true><<<(int)b->P.work[kColList].size(), COL_NT, G2::smem, b->stream>>>(
      maps, a, Geom{}, Coef<float>{});
  CKB(b, cudaGetLastError());
  b->cur = dst;
  b->launches++;
  return LKS_OK;
}

lks_status fwd_step(lks_batch* b, int t_new, bool jacc, float* tu, float* tv) {
  if (b->fwd_col) return fwd_col_step(b, t_new, jacc, tu, tv);
  switch (b->cfg) {
    case 0: return fwd_step_c<0>(b, t_new, jacc, tu, tv);
    case 1: return fwd_step_c<1>(b, t_new, jacc, tu, tv);
    case 2: return fwd_step_c<2>(b, t_new, jacc, tu, tv);
    default: return fwd_step_c<3>(b, t_new, jacc, tu, tv);
  }
}
// One adjoint step of every design on the warp-column kernel (one CTA per entry of
// work list kAdjColList).
lks_status adj_col_step(lks_batch* b, const float* u1, const float* v1, const float* u0, const float* v0,
                        int sens_flow) {
  constexpr int NF = acol_nf(false);
  const int src = b->acur, dst = 1 - b->acur;
  TmaMaps<NF> maps;
  lks_status st;
  const float* mat = af(b, b->P.L.mat, 0);
  const float* fsrc[NF] = {adp(b, src, 0), adp(b, src, 1), adp(b, src, 2), adp(b, src, 3), adp(b, src, 4),
                           adp(b, src, 5), u1, v1, u0, v0, mat + b->P.A, mat};  // ..., alpha, 1/(1+alpha)
  for (int f = 0; f < NF; ++f)
    if ((st = arena_map(b, fsrc[f], COL_BW, ACOL_BH, &maps.m[f])) != LKS_OK) return st;
  AdjColArgs a;
  std::memset(&a, 0, sizeof(a));
  for (int q = 0; q < 6; ++q) a.m0[q] = adp(b, dst, q);
  a.gamma = af(b, b->P.L.gamma);
  a.emap = reinterpret_cast<const float*>(b->ws + b->P.L.emap);
  a.sens = af(b, b->P.L.sens);
  a.sens_flow = sens_flow;
  a.status = dstatus(b);
  a.work = reinterpret_cast<const BatchTile*>(b->ws + b->P.L.work[kAdjColList]);
  a.designs = ddesigns(b);
  a.pitch = b->P.W;
  adj_col_kernel<false, true><<<(int)b->P.work[kAdjColList].size(), COL_NT, acol_smem_bytes(false), b->stream>>>(
      maps, a, Geom{}, Coef<float>{});
  CKB(b, cudaGetLastError());
  b->acur = dst;
  b->launches++;
  return LKS_OK;
}

lks_status adj_step(lks_batch* b, const float* u1, const float* v1, const float* u0, const float* v0, int sf) {
  if (b->adj_col) return adj_col_step(b, u1, v1, u0, v0, sf);
  switch (b->cfg) {
    case 0: return adj_step_c<0>(b, u1, v1, u0, v0, sf);
    case 1: return adj_step_c<1>(b, u1, v1, u0, v0, sf);
    case 2: return adj_step_c<2>(b, u1, v1, u0, v0, sf);
    default: return adj_step_c<3>(b, u1, v1, u0, v0, sf);
  }
}

dim3 per_design_grid(lks_batch* b, int bx = kEwBX) { return dim3(bx, b->n); }
int arena_grid(size_t n) { return lks_host::elementwise_blocks(n); }

lks_status snap_store(lks_batch* b, int idx) {
  const Plan& P = b->P;
  unsigned char* base = b->ws + P.L.snaps + (size_t)idx * 3 * P.A * P.snap_elem;
  if (P.snap_type == LKS_SNAP_F32) {
    CKB(b, cudaMemcpyAsync(base, stp(b, b->cur, 0), P.A * 3 * 4, cudaMemcpyDeviceToDevice, b->stream));
    return LKS_OK;
  }
  float* sc = reinterpret_cast<float*>(b->ws + P.L.scales) + (size_t)idx * 3 * b->n;
  CKB(b, cudaMemsetAsync(sc, 0, sizeof(float) * 3 * b->n, b->stream));
  for (int f = 0; f < 3; ++f) {
    const float* x = stp(b, b->cur, f);
    batch_absmax_kernel<<<per_design_grid(b), 256, 0, b->stream>>>(x, ddesigns(b), P.W, sc + f * b->n);
    unsigned char* y = base + (size_t)f * P.A * P.snap_elem;
    if (P.snap_type == LKS_SNAP_BF16)
      batch_encode_kernel<__nv_bfloat16><<<per_design_grid(b), 256, 0, b->stream>>>(
          x, reinterpret_cast<__nv_bfloat16*>(y), ddesigns(b), P.W, sc + f * b->n);
    else
      batch_encode_kernel<__half><<<per_design_grid(b), 256, 0, b->stream>>>(x, reinterpret_cast<__half*>(y),
                                                                              ddesigns(b), P.W, sc + f * b->n);
    b->launches += 2;
  }
  CKB(b, cudaGetLastError());
  return LKS_OK;
}

lks_status snap_load(lks_batch* b, int idx) {
  const Plan& P = b->P;
  const unsigned char* base = b->ws + P.L.snaps + (size_t)idx * 3 * P.A * P.snap_elem;
  if (P.snap_type == LKS_SNAP_F32) {
    CKB(b, cudaMemcpyAsync(stp(b, b->cur, 0), base, P.A * 3 * 4, cudaMemcpyDeviceToDevice, b->stream));
    return LKS_OK;
  }
  const float* sc = reinterpret_cast<const float*>(b->ws + P.L.scales) + (size_t)idx * 3 * b->n;
  for (int f = 0; f < 3; ++f) {
    float* x = stp(b, b->cur, f);
    const unsigned char* y = base + (size_t)f * P.A * P.snap_elem;
    if (P.snap_type == LKS_SNAP_BF16)
      batch_decode_kernel<__nv_bfloat16><<<per_design_grid(b), 256, 0, b->stream>>>(
          reinterpret_cast<const __nv_bfloat16*>(y), x, ddesigns(b), P.W, sc + f * b->n);
    else
      batch_decode_kernel<__half><<<per_design_grid(b), 256, 0, b->stream>>>(reinterpret_cast<const __half*>(y), x,
                                                                              ddesigns(b), P.W, sc + f * b->n);
    b->launches++;
  }
  CKB(b, cudaGetLastError());
  return LKS_OK;
}

lks_status flush(lks_batch* b) {
  flush_accum_kernel<float><<<arena_grid(b->P.A), 256, 0, b->stream>>>(
      af(b, b->P.L.sens), reinterpret_cast<double*>(b->ws + b->P.L.sens64), b->P.A);
  CKB(b, cudaGetLastError());
  b->launches++;
  return LKS_OK;
}

lks_status materials(lks_batch* b) {
  float* m = af(b, b->P.L.mat, 0);
  batch_material_kernel<<<per_design_grid(b), 256, 0, b->stream>>>(af(b, b->P.L.gamma), ddesigns(b), b->P.W, m,
                                                                     m + b->P.A);
  CKB(b, cudaGetLastError());
  b->launches++;
  return LKS_OK;
}

// Every step of one batched gradient, enqueued on b->stream (captured once when a
// graph is used).  Reads the gamma pointer table, writes J to jval and the
// gradients through the output pointer table.
lks_status enqueue_gradient(lks_batch* b) {
  const Plan& P = b->P;
  const BLayout& L = P.L;
  const size_t A = P.A, fb = A * 4;
  const int n = P.n_steps, K = P.K;
  lks_status st;
  scatter_gamma_kernel<<<per_design_grid(b), 256, 0, b->stream>>>(
      reinterpret_cast<const float* const*>(b->ws + L.gptr), af(b, L.gamma), ddesigns(b), P.W);
  CKB(b, cudaGetLastError());
  b->launches++;
  if ((st = materials(b)) != LKS_OK) return st;
  CKB(b, cudaMemsetAsync(b->ws + L.stA, 0, fb * 3, b->stream));
  CKB(b, cudaMemsetAsync(b->ws + L.status, 0, sizeof(int), b->stream));
  const int flist = b->fwd_col ? kColList : b->cfg;  // work list of the forward (J partials per tile)
  CKB(b, cudaMemsetAsync(b->ws + L.jt, 0, sizeof(double) * P.work[flist].size(), b->stream));
  b->cur = 0;
  // forward march with a snapshot every K steps (Step 2), J accumulated per step (Step 3)
  for (int t = 0; t < n; ++t) {
    if (t % K == 0 && (st = snap_store(b, t / K)) != LKS_OK) return st;
    if ((st = fwd_step(b, t + 1, t >= 1, nullptr, nullptr)) != LKS_OK) return st;
  }
  batch_objective_kernel<NTHREADS><<<per_design_grid(b, kJBX), NTHREADS, 0, b->stream>>>(
      stp(b, b->cur, 1), stp(b, b->cur, 2), af(b, L.gamma), ddesigns(b), P.W,
      reinterpret_cast<double*>(b->ws + L.jfin));
  batch_reduce_J_kernel<<<b->n, NTHREADS, 0, b->stream>>>(
      reinterpret_cast<const double*>(b->ws + L.jt), reinterpret_cast<const int*>(b->ws + L.rng[flist]),
      reinterpret_cast<const double*>(b->ws + L.jfin), kJBX, reinterpret_cast<double*>(b->ws + L.jval));
  CKB(b, cudaGetLastError());
  b->launches += 2;
  // checkpointed adjoint (Step 4) with the sensitivity accumulated per level (Step 5)
  CKB(b, cudaMemsetAsync(b->ws + L.adA, 0, fb * 6, b->stream));
  CKB(b, cudaMemsetAsync(b->ws + L.sens, 0, fb, b->stream));
  CKB(b, cudaMemsetAsync(b->ws + L.sens64, 0, A * 8, b->stream));
  b->acur = 0;
  int since_flush = 0;
  auto store = [&](int s) { return af(b, (s & 1) ? L.seg2 : L.seg); };
  // segment s recomputed from its snapshot into store s & 1
  auto recompute = [&](int s) -> lks_status {
    const int t_lo = s * K, t_hi = std::min((s + 1) * K, n), top = std::min(t_hi + 1, n);
    float* seg = store(s);
    lks_status rs;
    b->cur = 0;
    if ((rs = snap_load(b, s)) != LKS_OK) return rs;
    CKB(b, cudaMemcpyAsync(seg, stp(b, b->cur, 1), fb, cudaMemcpyDeviceToDevice, b->stream));
    CKB(b, cudaMemcpyAsync(seg + A, stp(b, b->cur, 2), fb, cudaMemcpyDeviceToDevice, b->stream));
    for (int t = t_lo; t < top; ++t) {
      float* p = seg + (size_t)(t + 1 - t_lo) * 2 * A;
      if ((rs = fwd_step(b, t + 1, false, p, p + A)) != LKS_OK) return rs;
    }
    return LKS_OK;
  };
  // the adjoint steps over segment s
  auto march = [&](int s) -> lks_status {
    const int t_lo = s * K, t_hi = std::min((s + 1) * K, n);
    const float* seg = store(s);
    lks_status ms;
    const int t_stop = (s == 0) ? 1 : t_lo + 1;
    for (int t = t_hi; t >= t_stop; --t) {
      const float* l1 = seg + (size_t)(std::min(t + 1, n) - t_lo) * 2 * A;
      const float* l0 = seg + (size_t)(t - t_lo) * 2 * A;
      if ((ms = adj_step(b, l1, l1 + A, l0, l0 + A, t >= 1)) != LKS_OK) return ms;
      if (++since_flush == kFlushEvery) {
        if ((ms = flush(b)) != LKS_OK) return ms;
        since_flush = 0;
      }
    }
    return LKS_OK;
  };
  // Segment s - 1 is recomputed on the second stream while the adjoint marches
  // segment s; the adjoint waits for its segment's recompute, a recompute for the
  // adjoint that last read its store, and the last recompute (segment 0) is waited
  // for before the last adjoint, so the second stream ends joined.
  const int last = P.n_ckpt - 1;
  // On every exit, error paths included, the stream is restored and made to wait for
  // whatever the second stream holds (inside a capture this is the join).
  struct Restore {
    lks_batch* b;
    cudaStream_t s;
    ~Restore() {
      b->stream = s;
      if (cudaEventRecord(b->ev_fork, b->aux) == cudaSuccess) cudaStreamWaitEvent(s, b->ev_fork, 0);
    }
  } restore{b, b->stream};
  const cudaStream_t main = b->stream;
  CKB(b, cudaEventRecord(b->ev_fork, main));
  CKB(b, cudaStreamWaitEvent(b->aux, b->ev_fork, 0));
  b->stream = b->aux;
  if ((st = recompute(last)) != LKS_OK) return st;
  CKB(b, cudaEventRecord(b->ev_seg[last & 1], b->aux));
  for (int s = last; s >= 0; --s) {
    b->stream = main;
    CKB(b, cudaStreamWaitEvent(main, b->ev_seg[s & 1], 0));
    if (s > 0) {
      b->stream = b->aux;
      if (s < last) CKB(b, cudaStreamWaitEvent(b->aux, b->ev_adj[(s + 1) & 1], 0));
      if ((st = recompute(s - 1)) != LKS_OK) return st;
      CKB(b, cudaEventRecord(b->ev_seg[(s - 1) & 1], b->aux));
      b->stream = main;
    }
    if ((st = march(s)) != LKS_OK) return st;
    CKB(b, cudaEventRecord(b->ev_adj[s & 1], main));
  }
  if ((st = flush(b)) != LKS_OK) return st;
  gather_grad_kernel<<<per_design_grid(b), 256, 0, b->stream>>>(
      reinterpret_cast<const double*>(b->ws + L.sens64), reinterpret_cast<float* const*>(b->ws + L.dptr),
      ddesigns(b), P.W);
  CKB(b, cudaGetLastError());
  b->launches++;
  return LKS_OK;
}

// Times `steps` forward and adjoint steps of tile shape c on a uniform design (the
// forward / adjoint on the warp-column kernels when col / acol): us per forward and
// per adjoint step.
lks_status time_cfg(lks_batch* b, int c, bool col, bool acol, int steps, float* fwd_us, float* adj_us) {
  b->cfg = c;
  b->fwd_col = col;
  b->adj_col = acol;
  const size_t fb = b->P.A * 4;
  CKB(b, cudaMemsetAsync(b->ws + b->P.L.stA, 0, fb * 3, b->stream));
  CKB(b, cudaMemsetAsync(b->ws + b->P.L.adA, 0, fb * 6, b->stream));
  b->cur = 0;
  b->acur = 0;
  cudaEvent_t e[3];
  for (auto& x : e) CKB(b, cudaEventCreate(&x));
  lks_status st = LKS_OK;
  auto run = [&](int k) -> lks_status {
    lks_status s2;
    for (int q = 0; q < k; ++q)
      if ((s2 = fwd_step(b, 1 + q, false, nullptr, nullptr)) != LKS_OK) return s2;
    const float* u = stp(b, b->cur, 1);
    const float* v = stp(b, b->cur, 2);
    for (int q = 0; q < k; ++q)
      if ((s2 = adj_step(b, u, v, u, v, 1)) != LKS_OK) return s2;
    return LKS_OK;
  };
  // forward steps as a gradient runs them: half of them accumulate the objective
  // partials (the march), half store the level's u, v in the segment buffer (the
  // recompute)
  float* seg = af(b, b->P.L.seg);
  auto fwd_as_used = [&](int q) {
    if (q % 2 == 0) return fwd_step(b, 4 + q, true, nullptr, nullptr);
    float* lv = seg + (size_t)(1 + (q / 2) % (b->P.seg_levels - 1)) * 2 * b->P.A;
    return fwd_step(b, 4 + q, false, lv, lv + b->P.A);
  };
  if ((st = run(3)) == LKS_OK) {
    cudaEventRecord(e[0], b->stream);
    for (int q = 0; q < steps && st == LKS_OK; ++q) st = fwd_as_used(q);
    cudaEventRecord(e[1], b->stream);
    const float* u = stp(b, b->cur, 1);
    const float* v = stp(b, b->cur, 2);
    for (int q = 0; q < steps && st == LKS_OK; ++q) st = adj_step(b, u, v, u, v, 1);
    cudaEventRecord(e[2], b->stream);
  }
  if (st == LKS_OK) {
    cudaError_t ce = cudaEventSynchronize(e[2]);
    float m1 = 0.f, m2 = 0.f;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&m1, e[0], e[1]);
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&m2, e[1], e[2]);
    if (ce != cudaSuccess) st = bfail(b, LKS_ERR_CUDA, std::string("autotune timing: ") + cudaGetErrorString(ce));
    *fwd_us = m1 * 1000.f / (float)steps;
    *adj_us = m2 * 1000.f / (float)steps;
  }
  for (auto& x : e) cudaEventDestroy(x);
  return st;
}

lks_status autotune(lks_batch* b) {
  fill_gamma_kernel<<<per_design_grid(b), 256, 0, b->stream>>>(0.5f, af(b, b->P.L.gamma), ddesigns(b), b->P.W);
  CKB(b, cudaGetLastError());
  lks_status st;
  if ((st = materials(b)) != LKS_OK) return st;
  // A gradient runs two forward steps (march, recompute) and one adjoint step per
  // level.  tune_us[c]: that per-level time of tile shape c with its TMA kernels;
  // tune_col_us / tune_acol_us: a forward / adjoint step of the warp-column kernels.
  // The tile shape and the forward and adjoint kernels with the least per-level
  // time win (within what the options fix).
  const int shape_given = b->opt.tile_config;
  float adj_us[kNCfg] = {};
  for (int c = 0; c < kNCfg; ++c) {
    if (shape_given >= 0 && c != shape_given) continue;
    float fu = 0.f, au = 0.f;
    if ((st = time_cfg(b, c, false, false, 8, &fu, &au)) != LKS_OK) return st;
    b->tune_fwd_us[c] = fu;
    adj_us[c] = au;
    b->tune_us[c] = 2.f * fu + au;
  }
  b->tune_col_us = b->tune_acol_us = 0.f;
  if (b->opt.fwd_column != 0 || b->opt.adj_column != 0) {
    float fu = 0.f, au = 0.f;
    if ((st = time_cfg(b, shape_given >= 0 ? shape_given : 0, true, true, 8, &fu, &au)) != LKS_OK) return st;
    if (b->opt.fwd_column != 0) b->tune_col_us = fu;
    if (b->opt.adj_column != 0) b->tune_acol_us = au;
  }
  auto allowed = [](int option, int col) { return option < 0 || option == col; };
  int best = -1;
  bool best_col = false, best_acol = false;
  float best_us = 0.f;
  for (int c = 0; c < kNCfg; ++c) {
    if (shape_given >= 0 && c != shape_given) continue;
    for (int col = 0; col < 2; ++col)
      for (int acol = 0; acol < 2; ++acol) {
        if (!allowed(b->opt.fwd_column, col) || !allowed(b->opt.adj_column, acol)) continue;
        const float us = 2.f * (col ? b->tune_col_us : b->tune_fwd_us[c]) + (acol ? b->tune_acol_us : adj_us[c]);
        if (best < 0 || us < best_us) {
          best = c;
          best_col = col == 1;
          best_acol = acol == 1;
          best_us = us;
        }
      }
  }
  b->cfg = best;
  b->fwd_col = best_col;
  b->adj_col = best_acol;
  int dev_status = 0;
  CKB(b, cudaMemcpy(&dev_status, dstatus(b), sizeof(int), cudaMemcpyDeviceToHost));
  if (dev_status != 0) return bfail(b, (lks_status)dev_status, "device status raised while autotuning");
  return LKS_OK;
}

lks_status capture_graph(lks_batch* b) {
  cudaStream_t cap = nullptr;
  CKB(b, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cudaStream_t keep = b->stream;
  b->stream = cap;
  const int64_t l0 = b->launches;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  lks_status st = e == cudaSuccess ? enqueue_gradient(b) : LKS_ERR_CUDA;
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(cap, &g) : e;
  b->stream = keep;
  cudaStreamDestroy(cap);
  if (st != LKS_OK) {
    if (g) cudaGraphDestroy(g);
    return b->err.empty() ? bfail(b, st, "graph capture failed") : st;
  }
  if (e2 != cudaSuccess) return bfail(b, LKS_ERR_CUDA, std::string("stream capture: ") + cudaGetErrorString(e2));
  cudaGraphExec_t x = nullptr;
  const cudaError_t e3 = cudaGraphInstantiate(&x, g, 0);
  if (e3 != cudaSuccess) {
    cudaGraphDestroy(g);
    return bfail(b, LKS_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e3));
  }
  b->graph = g;
  b->exec = x;
  b->launches_per_grad = b->launches - l0;
  b->launches = l0;
  return LKS_OK;
}

}  // namespace

extern "C" {

lks_status lks_batch_workspace_size(int32_t n, const lks_problem_desc* descs, const lks_batch_options* opt,
                                    size_t* bytes) {
  if (!bytes) return LKS_ERR_INVALID_ARG;
  const lks_batch_options o = opt ? *opt : default_options();
  Plan P;
  const lks_status st = make_plan(n, descs, &o, &P, nullptr);
  if (st != LKS_OK) return st;
  *bytes = P.L.total;
  return LKS_OK;
}

lks_status lks_batch_create(int32_t n, const lks_problem_desc* descs, const lks_batch_options* opt, void* workspace,
                            size_t bytes, void* stream, lks_batch** out) {
  if (!out) return LKS_ERR_INVALID_ARG;
  *out = nullptr;
  lks_batch* b = new (std::nothrow) lks_batch();
  if (!b) return LKS_ERR_WORKSPACE;
  b->opt = opt ? *opt : default_options();
  std::string why;
  lks_status st = make_plan(n, descs, &b->opt, &b->P, &why);
  if (st != LKS_OK) {
    delete b;
    return st;
  }
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0 || bytes < b->P.L.total) {
    delete b;
    return LKS_ERR_WORKSPACE;
  }
  if (!encode_fn()) {  // the tensor-map encoder of the CUDA driver is required
    delete b;
    return LKS_ERR_CUDA;
  }
  b->n = n;
  b->d.assign(descs, descs + n);
  b->ws = static_cast<unsigned char*>(workspace);
  b->ws_bytes = bytes;
  b->stream = static_cast<cudaStream_t>(stream);
  auto fin = [&](lks_status s) {
    if (s != LKS_OK) {
      delete b;
      return s;
    }
    *out = b;
    return LKS_OK;
  };
  if (cudaGetDevice(&b->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess)
    return fin(LKS_ERR_CUDA);
  {
    bool ok = cudaStreamCreateWithFlags(&b->aux, cudaStreamNonBlocking) == cudaSuccess;
    for (cudaEvent_t* e : {&b->ev_fork, &b->ev_seg[0], &b->ev_seg[1], &b->ev_adj[0], &b->ev_adj[1]})
      ok = ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) return fin(LKS_ERR_CUDA);
  }
  const Plan& P = b->P;
  // per-design tables
  std::vector<BatchDesign> dz(n);
  std::vector<float> uin((size_t)n * (P.n_steps + 1)), emap((size_t)n * 540);
  for (int d = 0; d < n; ++d) {
    dz[d].g = make_geom(descs[d]);
    dz[d].c = make_coef<float>(descs[d]);
    dz[d].ax = P.ax[d];
    dz[d].ay = P.ay[d];
    for (int t = 0; t <= P.n_steps; ++t) uin[(size_t)t * n + d] = (float)inlet_amp(descs[d], t);
    const double A = (1.0 / 6.0 - descs[d].nu) * 4.5;
    double m[60];
    for (int cls = 0; cls < 9; ++cls) {
      flow_moment_map(A, cls, m);
      for (int q = 0; q < 60; ++q) emap[(size_t)d * 540 + cls * 60 + q] = (float)m[q];
    }
  }
  auto up_h = [&](size_t off, const void* src, size_t nb) {
    return cudaMemcpyAsync(b->ws + off, src, nb, cudaMemcpyHostToDevice, b->stream);
  };
  if (cudaMemsetAsync(b->ws, 0, P.L.total, b->stream) != cudaSuccess ||
      up_h(P.L.designs, dz.data(), sizeof(BatchDesign) * n) != cudaSuccess ||
      up_h(P.L.uin, uin.data(), sizeof(float) * uin.size()) != cudaSuccess ||
      up_h(P.L.emap, emap.data(), sizeof(float) * emap.size()) != cudaSuccess)
    return fin(bfail(b, LKS_ERR_CUDA, "upload of the design tables failed"));
  for (int c = 0; c < kNLists; ++c)
    if (up_h(P.L.work[c], P.work[c].data(), sizeof(BatchTile) * P.work[c].size()) != cudaSuccess ||
        up_h(P.L.rng[c], P.rng[c].data(), sizeof(int) * P.rng[c].size()) != cudaSuccess)
      return fin(bfail(b, LKS_ERR_CUDA, "upload of the work lists failed"));
  if ((st = setup_cfg<0>(b)) != LKS_OK || (st = setup_cfg<1>(b)) != LKS_OK || (st = setup_cfg<2>(b)) != LKS_OK ||
      (st = setup_cfg<3>(b)) != LKS_OK)
    return fin(st);
  if (cudaFuncSetAttribute(fwd_col2_kernel<C2_R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)Col2Geo<C2_R>::smem) != cudaSuccess ||
      cudaFuncSetAttribute(adj_col_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)acol_smem_bytes(false)) != cudaSuccess)
    return fin(bfail(b, LKS_ERR_CUDA, "shared-memory attributes of the column kernels"));
  if (b->opt.tile_config < 0 || b->opt.fwd_column < 0 || b->opt.adj_column < 0) {  // time what is not given
    if ((st = autotune(b)) != LKS_OK) return fin(st);
  } else {
    b->cfg = b->opt.tile_config;
    b->fwd_col = b->opt.fwd_column == 1;
    b->adj_col = b->opt.adj_column == 1;
  }
  if (b->opt.use_graph && (st = capture_graph(b)) != LKS_OK) return fin(st);
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return fin(bfail(b, LKS_ERR_CUDA, "create: sync failed"));
  return fin(LKS_OK);
}

lks_status lks_batch_gradient(lks_batch* b, const float* const* gamma_dev, double* J_dev, float* const* dJdgamma_dev) {
  if (!b || !gamma_dev || !J_dev || !dJdgamma_dev) return LKS_ERR_INVALID_ARG;
  const lks_host::Range range("lks_batch_gradient");
  for (int d = 0; d < b->n; ++d)
    if (!gamma_dev[d] || !dJdgamma_dev[d]) return bfail(b, LKS_ERR_INVALID_ARG, "NULL design pointer");
  const BLayout& L = b->P.L;
  CKB(b, cudaMemcpyAsync(b->ws + L.gptr, gamma_dev, sizeof(void*) * b->n, cudaMemcpyHostToDevice, b->stream));
  CKB(b, cudaMemcpyAsync(b->ws + L.dptr, dJdgamma_dev, sizeof(void*) * b->n, cudaMemcpyHostToDevice, b->stream));
  if (b->exec) {
    CKB(b, cudaGraphLaunch(b->exec, b->stream));
  } else {
    const int64_t l0 = b->launches;
    const lks_status st = enqueue_gradient(b);
    if (st != LKS_OK) return st;
    b->launches_per_grad = b->launches - l0;
  }
  CKB(b, cudaMemcpyAsync(J_dev, b->ws + L.jval, sizeof(double) * b->n, cudaMemcpyDeviceToDevice, b->stream));
  b->gradients++;
  return LKS_OK;
}

lks_status lks_batch_query(lks_batch* b, lks_batch_stats* out) {
  if (!b || !out) return LKS_ERR_INVALID_ARG;
  CKB(b, cudaStreamSynchronize(b->stream));
  int ds = 0;
  CKB(b, cudaMemcpy(&ds, dstatus(b), sizeof(int), cudaMemcpyDeviceToHost));
  std::memset(out, 0, sizeof(*out));
  out->n_designs = b->n;
  out->tile_config = b->cfg;
  out->checkpoint_every = b->P.K;
  out->n_ckpt = b->P.n_ckpt;
  out->arena_w = b->P.W;
  out->arena_h = b->P.H;
  out->graph = b->exec ? 1 : 0;
  out->device_status = ds;
  out->nodes = b->P.nodes;
  out->ntiles = (int64_t)b->P.work[b->cfg].size();
  out->workspace_bytes = (int64_t)b->P.L.total;
  out->kernel_launches = b->launches_per_grad;
  out->gradients = b->gradients;
  for (int c = 0; c < kNCfg; ++c) out->tune_us[c] = b->tune_us[c];
  out->fwd_column = b->fwd_col ? 1 : 0;
  for (int c = 0; c < kNCfg; ++c) out->tune_fwd_us[c] = b->tune_fwd_us[c];
  out->tune_col_us = b->tune_col_us;
  out->adj_column = b->adj_col ? 1 : 0;
  out->tune_acol_us = b->tune_acol_us;
  return LKS_OK;
}

lks_status lks_batch_destroy(lks_batch* b) {
  if (!b) return LKS_ERR_INVALID_ARG;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  delete b;
  return LKS_OK;
}

const char* lks_batch_last_error(const lks_batch* b) { return b ? b->err.c_str() : "null batch handle"; }

}  // extern "C"
