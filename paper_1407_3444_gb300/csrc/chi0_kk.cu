// chi0_kk.cu -- Re chi0 from Im chi0 by the Kramers-Kronig relation (the route the paper calls
// the usual one, Sec. II below Eqs. 1-3), the alternative to the principal value of Eq. 1.
//
// With Im odd in w (Eq. 3) and the positive-sign convention of this library,
//   Re(w) = (1/pi) PV int_0^inf Im(u) [1/(u - w) + 1/(u + w)] du.
// Im is known on a uniform grid u_j = j du, j < m (Im(0) = 0, Im = 0 from u_m on: the grid
// must cover the spectrum, the caveat of Sec. IV), and is taken piecewise linear between the
// nodes.  The hat function of node j integrates against 1/(u - w) to the second difference of
// G(x) = x ln|x| (G'' = 1/x, G(0) = 0):
//   int hat_j(u) / (u - w) du = [G(u_{j+1} - w) - 2 G(u_j - w) + G(u_{j-1} - w)] / du,
// finite also where w is a node.  Summing by parts over the nodes,
//   Re(w) = (1 / (pi du)) sum_{k=0..m} [G(u_k - w) + G(u_k + w)] (Im_{k-1} - 2 Im_k + Im_{k+1}),
// with Im_j = 0 for j <= 0 and j >= m.  One thread per output node, FP64, O(m) per node.
#include <cuda_runtime.h>
#include <math.h>

#include "chi0_internal.h"

namespace chi0int {
namespace {

__device__ __forceinline__ double gxl(double x) { return x == 0.0 ? 0.0 : x * log(fabs(x)); }

__global__ void __launch_bounds__(256) k_kk(const double *__restrict__ im, int m, double du, double scale,
                                            const double *__restrict__ dos, int ndos, double *__restrict__ re) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const double w = i * du;
  double s = 0.0, c = 0.0;  // compensated sum
  auto I = [&](int j) { return j >= 1 && j < m ? im[j] : 0.0; };  // Im(0) = 0; 0 past the grid
  for (int k = 0; k <= m; ++k) {
    const double d2 = I(k - 1) - 2.0 * I(k) + I(k + 1);
    if (d2 == 0.0) continue;
    const double uk = k * du;
    const double t = (gxl(uk - w) + gxl(uk + w)) * d2;
    const double y = s + t;
    c += fabs(s) >= fabs(t) ? (s - y) + t : (t - y) + s;
    s = y;
  }
  double v = (s + c) / (3.141592653589793 * du);
  if (dos && i == 0) {  // the q -> 0 intraband limit at w = 0 (Sec. III), as the direct route adds it
    double sd = 0.0;
    for (int k = 0; k < ndos; ++k) sd += dos[k];
    v += scale * sd;
  }
  re[i] = v;
}

}  // namespace

cudaError_t launch_kk(const double *im, int m, double du, double scale, const double *dos, int ndos, double *re,
                      cudaStream_t s) {
  if (m <= 1 || !(du > 0.0)) return cudaErrorInvalidValue;
  k_kk<<<(m + 255) / 256, 256, 0, s>>>(im, m, du, scale, dos, ndos, re);
  return cudaGetLastError();
}

}  // namespace chi0int
