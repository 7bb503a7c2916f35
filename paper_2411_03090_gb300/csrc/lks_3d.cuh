// lks_3d.cuh -- host interface of the three-dimensional (D3Q19) steady duct path,
// implemented in lks_3d.cu and driven by the handle code of lks_capi.cu.
//
// The scheme is the paper's LKS / ALKS (arXiv 2411.03090, Secs. 2.4-2.5, App. A)
// written for 19 velocities: the inlet face x = 0 carries a duct profile, the
// outlet face x = nx-1 a prescribed pressure, the four side faces are walls;
// nodes on two or three faces are wall nodes whose density is carried over from
// the neighbour one node inward along the side-wall normals.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/lks.h"

namespace lks3 {

// Workspace layout of a D3Q19 problem (byte offsets; fields of N = nx ny nz
// values of the real type, x fastest, then y, then z).
struct Layout3 {
  size_t N = 0, rsize = 4;
  size_t gamma = 0, stA = 0, stB = 0, adA = 0, adB = 0, binv = 0, src = 0;
  size_t jpart = 0, jval = 0, status = 0, emap = 0, total = 0;
  int jblocks = 0;
};

Layout3 make_layout3(const lks_problem_desc& d);

// Number of adjoint fields: rho~, u~ (3), s~ (xx, xy, xz, yy, yz, zz).
constexpr int kNA3 = 10;
// Edge classes: index (n_x + 1) * 9 + (n_y + 1) * 3 + (n_z + 1) of the outward
// normal (sum of the face normals); class 22 (n = (1, 0, 0)) is the outlet face.
constexpr int kClasses3 = 27;
// Per single face (axis a, outward sign s; index 2a + (s > 0)): the 5 x 5 fill of the
// unknown links from the opposite links, then the unknowns' boundary objective term.
constexpr int kFillLen3 = 30;

// Everything the 3-D marches need from the handle.
struct Ctx3 {
  const lks_problem_desc* d;
  const Layout3* L;
  unsigned char* ws;
  cudaStream_t stream;
  int64_t* launches;
  std::string* err;
};

// Uploads the host-built adjoint edge maps (kClasses3 x 10 x 19), the per-class
// boundary objective terms of the moments (kClasses3 x 10) and the six single-face
// fills (6 x kFillLen3).
lks_status upload_maps3(const Ctx3& c);
// Steps 2-3: gamma -> state after n_steps; J of the final state into J_dev (may be
// null).  *cur receives the buffer (0 = A, 1 = B) holding the final state, *path the
// lks_exec_path that ran (column: the warp-column forward, FP32 with nx % 4 == 0
// unless the step path is asked for).
lks_status forward3(const Ctx3& c, const void* gamma_dev, double* J_dev, int* cur, int* path);
// Step 4: n_adj ALKS iterations on the frozen state `cur`; *acur receives the
// adjoint buffer holding the result, *path the lks_exec_path that ran (column: the
// warp-column adjoint, under the same conditions as the forward's).
lks_status adjoint3(const Ctx3& c, int cur, int* acur, int* path);
// Step 5: dJ/dgamma of the final state and adjoint into out (N values).
lks_status sensitivity3(const Ctx3& c, int cur, int acur, void* out);

// Host-only: the 10 x 19 adjoint moment map of one edge class at parameter A
// (rows rho~, u~x, u~y, u~z, s~xx, s~xy, s~xz, s~yy, s~yz, s~zz; columns the 19
// gathered f~, zero for unknown links).  unit (10 values, may be null): the moments
// when every residual row carries a unit boundary objective term and the gathered
// f~ are zero (Eqs. afboundaryu / afboundaryp).  fill (kFillLen3 values, may be
// null; single faces only): the unknown links (c . n > 0, in link order) per unit of
// each opposite link (c . n < 0, in link order), 5 x 5 row-major, then the unknowns
// under a unit term in every row.  The rule's columns of the links with c . n = 0
// are zero, so these determine the unknowns.
void flow_moment_map3(double A, int cls, double* out, double* unit, double* fill = nullptr);

}  // namespace lks3
