// chi0_grid.cuh -- device helpers shared by the weight kernels: tetrahedron corners of the
// k mesh (Sec. II: the integration domain split into tetrahedra) at k and at k+q, small
// quotients without a division sequence, and warp sums.
#pragma once

#include <cuda_runtime.h>

#include "chi0_internal.h"

namespace chi0int {
namespace grid {

constexpr unsigned kFull = 0xffffffffu;

// x / d for 0 <= x < qmax * d (small quotients): binary search, no division sequence
__device__ __forceinline__ int div_small(int x, int d, int qmax) {
  int lo = 0, hi = qmax;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (mid * d <= x) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Corners of tetrahedron t at k and at k+q, and its fractional volume.  Builtin mesh:
// tetrahedron 6*cube + p = {000, e_a, e_a + e_b, 111} for the p-th axis order (a, b, .)
// of the lexicographically ordered permutations of (0, 1, 2).
__device__ __forceinline__ void tet_corners(const Grid &g, const Tet &tet, const Q &q, long long t,
                                            long long c[4], long long cq[4], double &vol) {
  if (tet.corners) {
    const int4 v = tet.corners[t];
    c[0] = v.x; c[1] = v.y; c[2] = v.z; c[3] = v.w;
    vol = tet.vol[t];
    for (int i = 0; i < 4; ++i) cq[i] = q.Eq ? c[i] : shift_corner(g, c[i], q.shift);
    return;
  }
  const unsigned tu = (unsigned)t;
  const unsigned cube = tu / 6u;
  const int p = (int)(tu - cube * 6u);
  const unsigned r = fdiv(cube, g.fn2);
  const int i2 = (int)(cube - r * (unsigned)g.n[2]);
  const unsigned i0u = fdiv(r, g.fn1);
  const int i1 = (int)(r - i0u * (unsigned)g.n[1]);
  const int i0 = (int)i0u;
  const int ax = p >> 1;                                // first axis: 0,0,1,1,2,2
  const int bx = (p == 0) ? 1 : (p == 1) ? 2 : (p == 2) ? 0 : (p == 3) ? 2 : (p == 4) ? 0 : 1;
  int o1[3] = {0, 0, 0}, o2[3] = {0, 0, 0};
  o1[ax] = 1;
  o2[ax] = 1;
  o2[bx] = 1;
  const int *s = q.shift;
  const bool ex = q.Eq != nullptr;
  c[0] = cid(g, i0, i1, i2);
  c[1] = cid(g, i0 + o1[0], i1 + o1[1], i2 + o1[2]);
  c[2] = cid(g, i0 + o2[0], i1 + o2[1], i2 + o2[2]);
  c[3] = cid(g, i0 + 1, i1 + 1, i2 + 1);
  if (ex) {
    for (int i = 0; i < 4; ++i) cq[i] = c[i];
  } else {
    cq[0] = cid(g, i0 + s[0], i1 + s[1], i2 + s[2]);
    cq[1] = cid(g, i0 + o1[0] + s[0], i1 + o1[1] + s[1], i2 + o1[2] + s[2]);
    cq[2] = cid(g, i0 + o2[0] + s[0], i1 + o2[1] + s[1], i2 + o2[2] + s[2]);
    cq[3] = cid(g, i0 + 1 + s[0], i1 + 1 + s[1], i2 + 1 + s[2]);
  }
  vol = tet.vol_builtin;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

}  // namespace grid
}  // namespace chi0int
