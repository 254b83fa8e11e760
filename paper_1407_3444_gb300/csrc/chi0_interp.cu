// chi0_interp.cu -- energies and eigenvectors at k+q for q off the k mesh, by linear
// interpolation from the mesh (Sec. II: the data at k+q, which are in general not on the
// tetrahedron mesh, are approximated by linear interpolation, energies and matrix elements on
// equal footing).
//
// For a corner k of the periodic mesh, k+q lies in one cube of the mesh and, within it, in one
// of the cube's six tetrahedra {000, e_p0, e_p0 + e_p1, 111} (the axis order p that sorts the
// local coordinates t descending, t_p0 >= t_p1 >= t_p2).  Its barycentric weights there are
//   (1 - t_p0, t_p0 - t_p1, t_p1 - t_p2, t_p2),
// and every quantity is the weighted sum of its values at those four corners, band by band.
// Eigenvectors carry an arbitrary phase per corner, so before the sum the vectors of corners
// 1..3 are turned onto the phase of corner 0's (multiplied by conj(<v_0|v_i>) / |<v_0|v_i>|),
// and the sum is normalised.  |M_mn|^2 does not depend on the phase left over.
#include <cuda_runtime.h>
#include <math.h>

#include "chi0_internal.h"

namespace chi0int {
namespace {

struct Cd {
  double x, y;
};
__device__ __forceinline__ Cd ld(const void *C, int dtype, long long i) {
  if (dtype == 0) {  // complex64
    const float2 v = ((const float2 *)C)[i];
    return Cd{v.x, v.y};
  }
  const double2 v = ((const double2 *)C)[i];
  return Cd{v.x, v.y};
}
__device__ __forceinline__ void st(void *C, int dtype, long long i, Cd v) {
  if (dtype == 0) ((float2 *)C)[i] = make_float2((float)v.x, (float)v.y);
  else ((double2 *)C)[i] = make_double2(v.x, v.y);
}

// one thread per (corner, band)
__global__ void __launch_bounds__(256) k_interp_kq(Grid g, const double *__restrict__ E, const void *__restrict__ C,
                                                   int dtype, double q0, double q1, double q2,
                                                   double *__restrict__ Eq, void *__restrict__ Cq) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= g.nc * g.nb) return;
  const long long c = idx / g.nb;
  const int b = (int)(idx - c * g.nb);
  const int i2 = (int)(c % g.N[2]), i1 = (int)((c / g.N[2]) % g.N[1]), i0 = (int)(c / ((long long)g.N[2] * g.N[1]));
  const int ii[3] = {i0, i1, i2};
  const double qq[3] = {q0, q1, q2};
  int base[3];
  double t[3];
  for (int d = 0; d < 3; ++d) {
    const double x = ii[d] + qq[d] * g.n[d];
    const double fl = floor(x);
    t[d] = x - fl;
    long long m = (long long)fl % g.n[d];
    if (m < 0) m += g.n[d];
    base[d] = (int)m;
  }
  // axis order sorting t descending (ties: lower axis first)
  int p0 = 0, p1 = 1, p2 = 2;
  if (t[p1] > t[p0]) { const int s = p0; p0 = p1; p1 = s; }
  if (t[p2] > t[p1]) { const int s = p1; p1 = p2; p2 = s; }
  if (t[p1] > t[p0]) { const int s = p0; p0 = p1; p1 = s; }
  const double w[4] = {1.0 - t[p0], t[p0] - t[p1], t[p1] - t[p2], t[p2]};
  long long cc[4];
  int o[3] = {0, 0, 0};
  for (int v = 0; v < 4; ++v) {
    if (v == 1) o[p0] = 1;
    if (v == 2) o[p1] = 1;
    if (v == 3) o[p2] = 1;
    const int j0 = (base[0] + o[0]) % g.n[0], j1 = (base[1] + o[1]) % g.n[1], j2 = (base[2] + o[2]) % g.n[2];
    cc[v] = ((long long)j0 * g.N[1] + j1) * g.N[2] + j2;
  }
  double e = 0.0;
  for (int v = 0; v < 4; ++v) e += w[v] * E[cc[v] * g.nb + b];
  Eq[c * g.nb + b] = e;
  if (!C) return;
  // phases of corners 1..3 relative to corner 0: <v_0|v_i>
  Cd ph[4] = {{1.0, 0.0}, {1.0, 0.0}, {1.0, 0.0}, {1.0, 0.0}};
  for (int v = 1; v < 4; ++v) {
    double re = 0.0, im = 0.0;
    for (int o = 0; o < g.norb; ++o) {
      const Cd a = ld(C, dtype, (cc[0] * g.norb + o) * g.nb + b), z = ld(C, dtype, (cc[v] * g.norb + o) * g.nb + b);
      re += a.x * z.x + a.y * z.y;
      im += a.x * z.y - a.y * z.x;
    }
    const double m = sqrt(re * re + im * im);
    if (m > 0.0) ph[v] = Cd{re / m, -im / m};  // conj(<v_0|v_i>) / |.|
  }
  double nrm = 0.0;
  for (int o = 0; o < g.norb; ++o) {
    double sx = 0.0, sy = 0.0;
    for (int v = 0; v < 4; ++v) {
      const Cd z = ld(C, dtype, (cc[v] * g.norb + o) * g.nb + b);
      sx += w[v] * (z.x * ph[v].x - z.y * ph[v].y);
      sy += w[v] * (z.x * ph[v].y + z.y * ph[v].x);
    }
    nrm += sx * sx + sy * sy;
  }
  const double sc = nrm > 0.0 ? 1.0 / sqrt(nrm) : 0.0;
  for (int o = 0; o < g.norb; ++o) {
    double sx = 0.0, sy = 0.0;
    for (int v = 0; v < 4; ++v) {
      const Cd z = ld(C, dtype, (cc[v] * g.norb + o) * g.nb + b);
      sx += w[v] * (z.x * ph[v].x - z.y * ph[v].y);
      sy += w[v] * (z.x * ph[v].y + z.y * ph[v].x);
    }
    st(Cq, dtype, (c * g.norb + o) * g.nb + b, Cd{sx * sc, sy * sc});
  }
}

}  // namespace

cudaError_t launch_interp_kq(const Grid &g, const double *E, const void *C, int c64, const double q[3], double *Eq,
                             void *Cq, cudaStream_t s) {
  const long long n = g.nc * g.nb;
  k_interp_kq<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, E, C, c64 ? 0 : 1, q[0], q[1], q[2], Eq, Cq);
  return cudaGetLastError();
}

}  // namespace chi0int
