// Host build of the CUDA path's per-tetrahedron arithmetic (paper_1407_3444_gb300/csrc/
// chi0_math.cuh) for CPU regression tests against the FP64 oracle between GPU runs.  The
// device qualifiers become plain inline functions; the three CUDA intrinsics the header
// calls get host stand-ins (correctly rounded reciprocal and quotient; log2).  The functions
// below follow the weight kernels' use of the header for one tetrahedron and one band pair:
// the static kernel's series / queued-table split (Eq. 1 at w = 0) and the dynamic kernel's
// mixed path (offset carving, far-field moments, near-field table, B-spline Im; Eqs. 1-2).
// Host rounding differs from the GPU's (FMA contraction), so they are compared at the
// mixed-precision tolerance, not bitwise.
#include <algorithm>
#include <cmath>
#include <cstring>
using std::max;
using std::min;
#define __device__
#define __forceinline__ inline
#define __noinline__ __attribute__((noinline))
#define __constant__
#define __log2f log2f
#define __frcp_rn(x) (1.0f / (x))
#define __fdividef(a, b) ((a) / (b))
#include "../../paper_1407_3444_gb300/csrc/chi0_math.cuh"

using namespace chi0dev;

namespace {
constexpr float kTau = 9.5367431640625e-07f;  // 2^-20, the library default

// a final tetrahedron of the static path: the kernel's series, else its queued evaluation
template <typename T> double static_piece(T r, T d[4], T ff[4]) {
  sort4(d, ff);
  if (series_ok(d, T(Num<T>::kappa))) return (double)(r * series_sum(d, ff));
  if constexpr (sizeof(T) == 8) {
    return r * inv_sum_table(d, ff);
  } else {
    float x[4];
    if (!mixed_knots(x, d, kTau)) return (double)(r * inv_sum_long(x, ff));
    double t = 0.0, xd[4] = {x[0], x[1], x[2], x[3]}, fd[4] = {ff[0], ff[1], ff[2], ff[3]};
    for (int j = 0; j < 4; ++j) t += inv_term_table(xd, fd, j);
    return (double)r * t;
  }
}
}  // namespace

// (1/V) int_{a<0<b} 2 f / D over one tetrahedron (corner values a = e_k - eF, b = e_{k+q} - eF)
extern "C" double host_static(const double *a64, const double *b64, const double *f64, int fp64) {
  double acc = 0.0;
  if (fp64) {
    double a[4], b[4], f[4];
    for (int i = 0; i < 4; ++i) a[i] = a64[i], b[i] = b64[i], f[i] = f64[i];
    carve2<double>(a, b, f, [&](double r, double d[4], double ff[4]) { acc += static_piece<double>(r, d, ff); });
  } else {
    float a[4], b[4], f[4];
    for (int i = 0; i < 4; ++i) a[i] = (float)a64[i], b[i] = (float)b64[i], f[i] = (float)f64[i];
    carve2<float>(a, b, f, [&](float r, float d[4], float ff[4]) { acc += static_piece<float>(r, d, ff); });
  }
  return 2.0 * acc;
}

// (1/V) int f [1/(D - w) + 1/(D + w)] (PV) and pi (1/V) int f delta(w - D) on nw frequencies
// w >= 0, the dynamic kernel's mixed path (FP32 energies as hi + lo pairs)
extern "C" void host_dynamic_mixed(const double *a64, const double *b64, const double *f64, int nw,
                                   const double *w, double *re, double *im) {
  float a[4], al[4], bh[4], bl[4], f[4], e[4];
  for (int i = 0; i < 4; ++i) {
    a[i] = (float)a64[i];
    al[i] = (float)(a64[i] - (double)a[i]);
    bh[i] = (float)b64[i];
    bl[i] = (float)(b64[i] - (double)bh[i]);
    f[i] = (float)f64[i];
  }
  float sv, tv;
  two_diff(bh[0], a[0], sv, tv);
  const float corr = tv + (bl[0] - al[0]);
  const float D0h = sv + corr, D0l = corr - (D0h - sv);
  e[0] = 0.0f;
  for (int i = 1; i < 4; ++i) {
    float sa, ta, sb, tb;
    two_diff(a[i], a[0], sa, ta);
    two_diff(bh[i], bh[0], sb, tb);
    e[i] = (sb - sa) + ((tb - ta) + ((bl[i] - bl[0]) - (al[i] - al[0])));
  }
  for (int k = 0; k < nw; ++k) re[k] = im[k] = 0.0;
  carve2_off<float>(a, e, D0h, f, [&](float r, float ee[4], float ff[4]) {
    sort4(ee, ff);
    float d[4];
    for (int i = 0; i < 4; ++i) d[i] = D0h + ee[i];
    if (!(d[3] > 0.0f)) return;
    float am[32];
    const int K = far_moments<float, 32>(d, ff, am);
    const float c = D0h + (ee[0] + ee[3]) * 0.5f, half = (ee[3] - ee[0]) * 0.5f;
    int nf = 0;
    for (int k = 0; k < nw; ++k) {
      const float wh = (float)w[k], wl = (float)(w[k] - (double)wh);
      const float om = wh;
      float rr = 0.0f;
      const float rp = half / (c + om);
      if (rp <= Num<float>::kappa_far) {
        rr += far_eval(am, K, c, -om, rp);
      } else {
        float x[4] = {d[0] + om, d[1] + om, d[2] + om, d[3] + om};
        rr += inv_sum_mixed(x, ff, kTau, &nf);
      }
      float sh, t2;
      two_diff(D0h, om, sh, t2);
      sh = sh + (t2 + (D0l - wl));
      float x[4] = {sh + ee[0], sh + ee[1], sh + ee[2], sh + ee[3]};
      const float dm = c - om, rm = half / (dm < 0.0f ? -dm : dm);
      if (rm <= Num<float>::kappa_far) rr += far_eval(am, K, c, om, rm);
      else rr += inv_sum_mixed(x, ff, kTau, &nf);
      re[k] += (double)(r * rr);
      if (rm > Num<float>::kappa_far && x[0] < 0.0f && x[3] > 0.0f)
        im[k] += (double)(r * (delta_sum(x, ff, 0.0f) * 3.141592653589793f));
    }
  });
}
