// chi0_math.cuh -- device arithmetic of the doubly carved linear tetrahedron method.
//
// Sec. II of Heil et al. (arXiv:1407.3444): the integrand of Eqs. 1-2 is restricted to
// the region where Th(eF - e^m_k) Th(e^n_{k+q} - eF) = 1 (Eq. 4) by cutting every
// tetrahedron twice, first by a = e^m_k - eF < 0, then by b = e^n_{k+q} - eF > 0.  On
// each final tetrahedron S (volume V, vertex values d_j = b_j - a_j >= 0 of
// D = e^n_{k+q} - e^m_k and f_j of |M|^2) the integrals are exact for the linear
// interpolants (Hermite-Genocchi):
//   (1/V) int_S lambda_j / (D - x)   = g[d_1-x, .., d_4-x, d_j-x],  g(t) = t^3 ln|t|
//   (1/V) int_S lambda_j delta(w - D) = M(w; d_1..d_4, d_j) / 4     (cubic B-spline density)
// with g[...] the fourth divided difference (knot d_j repeated).  The paper does not print
// its formulas; these are the closed forms for linear integrands on a simplex.
//
// Evaluation strategy (GPU-first; all branches exact up to rounding):
//  * knots clustered away from 0 (spread <= RHO * |nearest|): one Taylor series about
//    the mean for all four j at once (h_k complete homogeneous polynomials);
//  * otherwise the divided-difference table of the sorted knots, each entry by the
//    difference recursion or, where its own knots cluster, by its Taylor series;
//  * mixed precision: the table in FP32 only when every gap between sorted knots is at
//    least tau * max|knot|; below that (the near-degenerate, cancellation-prone case)
//    the table is evaluated in FP64.
#pragma once

#ifdef __CUDACC__
#include <cuda_runtime.h>
#endif
#include <math.h>
#include <stdint.h>

namespace chi0dev {

constexpr double kRho = 0.25;                     // Taylor branch threshold
constexpr double kFloor = 9.313225746154785e-10;  // 2^-30: >= 3 exactly-zero knots

template <typename T> struct Num;
template <> struct Num<double> {
  static __device__ __forceinline__ double lg(double x) { return log(x); }
  static constexpr double tol = 1e-17;
  static constexpr float log2_tol = -56.4727f;  // log2(tol)
  static constexpr double kappa = 0.25;  // series branch: (x3 - x0) <= kappa (x3 + x0)
  static constexpr double kappa_long = 0.25;
  static constexpr double kappa_far = 0.5;  // far-field expansion of the dynamic PV terms
  static constexpr int kmax = 80;
};
template <> struct Num<float> {
  static __device__ __forceinline__ float lg(float x) { return logf(x); }
  static constexpr float tol = 2e-8f;
  static constexpr float log2_tol = -25.5754f;  // log2(tol)
  static constexpr float kappa = 0.5f;       // series branch inside the carving loop
  static constexpr float kappa_long = 0.7f;  // series branch of queued pieces (evaluated together)
  static constexpr float kappa_far = 0.5f;   // far-field expansion of the dynamic PV terms
  static constexpr int kmax = 64;
};

template <typename T> __device__ __forceinline__ T tabs(T x) { return x < T(0) ? -x : x; }

// Reciprocal and quotient of the weight kernels.  FP64: IEEE division.  FP32: the hardware
// reciprocal approximation refined by one Newton-Raphson step, r' = r + r (1 - x r), within
// about 1 ulp of 1/x for normal x (0 and denormals are never divided by: ties and zero knots
// take their own branches), and the fast quotient (at most 2 ulp from a / b for the cut
// fractions, |b| < 2^126); both far below the FP32 path's 1e-6 target.  The correctly rounded
// intrinsics carry slow paths for special operands that made the weight kernels' hot code
// several times larger (instruction-cache misses).
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float rcp(float x) {
#ifdef __CUDA_ARCH__
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return fmaf(r, fmaf(-x, r, 1.0f), r);
#else
  return __frcp_rn(x);
#endif
}
__device__ __forceinline__ double quot(double a, double b) { return a / b; }
__device__ __forceinline__ float quot(float a, float b) { return __fdividef(a, b); }

template <typename T> __device__ __forceinline__ void cswap(T &x, T &y, T &fx, T &fy) {
  if (y < x) {
    T t = x; x = y; y = t;
    t = fx; fx = fy; fy = t;
  }
}

// ascending sort of 4 knots carrying their weights (5-comparator network)
template <typename T> __device__ __forceinline__ void sort4(T d[4], T f[4]) {
  cswap(d[0], d[1], f[0], f[1]);
  cswap(d[2], d[3], f[2], f[3]);
  cswap(d[0], d[2], f[0], f[2]);
  cswap(d[1], d[3], f[1], f[3]);
  cswap(d[1], d[2], f[1], f[2]);
}

// g(t) = t^3 ln|t|, g(0) = 0
template <typename T> __device__ __forceinline__ T g0(T t) {
  return t == T(0) ? T(0) : t * t * t * Num<T>::lg(tabs(t));
}

// g^(k)(c)/k! for k = 1..3 (c != 0)
template <typename T> __device__ __forceinline__ T glow(int k, T c, T L) {
  if (k == 1) return T(3) * c * c * L + c * c;
  if (k == 2) return (T(6) * c * L + T(5) * c) * T(0.5);
  return (T(6) * L + T(11)) * T(1.0 / 6.0);
}

// knot t[idx] for a compile-time sized register array without dynamic indexing
template <typename T> __device__ __forceinline__ T pick5(const T t[5], int idx) {
  T r = t[0];
  r = idx == 1 ? t[1] : r;
  r = idx == 2 ? t[2] : r;
  r = idx == 3 ? t[3] : r;
  r = idx == 4 ? t[4] : r;
  return r;
}

// 6 (-1)^m / ((m+4)(m+3)(m+2)(m+1)): coefficients of the Taylor series below (k = m + 4)
template <typename T, int N> struct TaylorCoef {
  T v[N];
  constexpr TaylorCoef() : v() {
    for (int m = 0; m < N; ++m) {
      const T c = T(6) / (T(m + 4) * T(m + 3) * T(m + 2) * T(m + 1));
      v[m] = (m & 1) ? -c : c;
    }
  }
};
__constant__ constexpr TaylorCoef<float, Num<float>::kmax + 4> kTayF{};
__constant__ constexpr TaylorCoef<double, Num<double>::kmax + 4> kTayD{};
template <typename T> __device__ __forceinline__ T taylor_coef(int m);
template <> __device__ __forceinline__ float taylor_coef<float>(int m) { return kTayF.v[m]; }
template <> __device__ __forceinline__ double taylor_coef<double>(int m) { return kTayD.v[m]; }

// Taylor series of the divided difference g[t_i..t_j] (n = j - i) of knots clustered about
// their mean c != 0, in the scaled offsets e = (t - c)/c (no powers of 1/c that could
// overflow):  g[t_i..t_j] = sum_{k=n}^{3} g^(k)(c)/k! c^(k-n) h_{k-n}(e)
//                        + c^(3-n) sum_{k>=4} 6 (-1)^(k-4) / (k(k-1)(k-2)(k-3)) h_{k-n}(e)
// with h_m the complete homogeneous symmetric polynomials.
template <typename T> __device__ __noinline__ T dd_taylor(const T t[5], int i, int j) {
  const int n = j - i;
  T c = T(0);
#pragma unroll
  for (int l = 0; l < 5; ++l) c += (l >= i && l <= j) ? t[l] : T(0);
  c = c / T(n + 1);
  const T ci = rcp(c);
  T e[5], h[5];
#pragma unroll
  for (int l = 0; l < 5; ++l) {
    e[l] = (l >= i && l <= j) ? (t[l] - c) * ci : T(0);  // padding variables are 0: no effect on h
    h[l] = T(1);
  }
  const T L = Num<T>::lg(tabs(c));
  T low = T(0), cp = T(1);  // cp = c^(k-n)
  for (int k = n; k < 4; ++k) {
    if (k > n) {
      h[0] = e[0] * h[0];
#pragma unroll
      for (int l = 1; l < 5; ++l) h[l] = h[l - 1] + e[l] * h[l];
      cp *= c;
    }
    low += (k == 0 ? g0(c) : glow(k, c, L)) * cp * h[4];
  }
  T high = T(0), prev = T(0), big = T(0);
  for (int k = 4; k < n + Num<T>::kmax; ++k) {
    if (k > n) {
      h[0] = e[0] * h[0];
#pragma unroll
      for (int l = 1; l < 5; ++l) h[l] = h[l - 1] + e[l] * h[l];
    }
    const T coef = taylor_coef<T>(k - 4);  // 6 (-1)^(k-4) / (k (k-1) (k-2) (k-3))
    const T term = coef * h[4];
    high += term;
    big = tabs(term) > big ? tabs(term) : big;
    if (k >= 5 && k - n >= 2 &&
        tabs(term) + tabs(prev) <= Num<T>::tol * (tabs(high) > big ? tabs(high) : big))
      break;
    prev = term;
  }
  T scale = T(1);  // c^(3-n)
  if (n == 4) scale = ci;
  else if (n == 2) scale = c;
  else if (n == 1) scale = c * c;
  return low + scale * high;
}

// Fourth divided difference g[t0..t4] of sorted knots (no 4 equal zeros).
template <typename T> __device__ T dd5(const T t[5]) {
  const T rho = T(kRho);
  T v[5];
#pragma unroll
  for (int l = 0; l < 5; ++l) v[l] = g0(t[l]);
#pragma unroll
  for (int n = 1; n <= 4; ++n) {
#pragma unroll
    for (int i = 0; i + n <= 4; ++i) {
      const int j = i + n;
      const T ti = t[i], tj = t[j];
      T r;
      if (ti == tj) {
        // all knots equal: g^(n)(t)/n!; at t = 0: 0 for n <= 2
        r = (ti == T(0)) ? T(0) : glow(n < 4 ? n : 3, ti, Num<T>::lg(tabs(ti)));
        if (n == 4) r = (ti == T(0)) ? T(0) : T(0.25) / ti;
      } else if ((ti > T(0) && tj - ti <= rho * ti) || (tj < T(0) && tj - ti <= rho * (-tj))) {
        r = dd_taylor(t, i, j);
      } else {
        r = (v[i + 1] - v[i]) / (tj - ti);
      }
      v[i] = r;
    }
  }
  return v[0];
}

// (-1)^k 6 k!/(k+4)! = (-1)^k 6/((k+1)(k+2)(k+3)(k+4)), the series coefficients below
template <typename T, int N> struct SeriesCoef {
  T v[N];
  constexpr SeriesCoef() : v() {
    for (int k = 0; k < N; ++k) {
      const T c = T(6) / (T(k + 1) * T(k + 2) * T(k + 3) * T(k + 4));
      v[k] = (k & 1) ? -c : c;
    }
  }
};
__constant__ constexpr SeriesCoef<float, Num<float>::kmax> kCoefF{};
__constant__ constexpr SeriesCoef<double, Num<double>::kmax> kCoefD{};
template <typename T> __device__ __forceinline__ T series_coef(int k);
template <> __device__ __forceinline__ float series_coef<float>(int k) { return kCoefF.v[k]; }
template <> __device__ __forceinline__ double series_coef<double>(int k) { return kCoefD.v[k]; }

// sum_j f_j (1/V) int_S lambda_j / X for sorted knots x of one sign with
// |x_i - c| <= kappa |c| about the midpoint c = (x_0 + x_3)/2:
// 1/(c (1 + lambda.e)), e = (x - c)/c, expanded in lambda.e:
//   (1/V) int lambda_j / X = (1/c) sum_k (-1)^k 6 k!/(k+4)! h_k(e_1..e_4, e_j)
template <typename T> __device__ T series_sum(const T x[4], const T f[4]) {
  const T c = (x[0] + x[3]) * T(0.5);
  const T ci = rcp(c);
  T e[4];
#pragma unroll
  for (int l = 0; l < 4; ++l) e[l] = (x[l] - c) * ci;
  T H[4] = {T(1), T(1), T(1), T(1)};  // H_k over the first l+1 variables
  T P[4] = {T(1), T(1), T(1), T(1)};  // h_k(e, e_j)
  T sum = T(0.25) * (f[0] + f[1] + f[2] + f[3]);  // k = 0: 6/24 sum_j f_j
  T prev = T(0), big = tabs(sum);
  for (int k = 1; k < Num<T>::kmax; ++k) {
    H[0] = e[0] * H[0];
#pragma unroll
    for (int l = 1; l < 4; ++l) H[l] = H[l - 1] + e[l] * H[l];
    T s = T(0);
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      P[jj] = H[3] + e[jj] * P[jj];
      s += f[jj] * P[jj];
    }
    const T term = series_coef<T>(k) * s;
    sum += term;
    big = tabs(term) > big ? tabs(term) : big;
    if (k >= 2 && tabs(term) + tabs(prev) <= Num<T>::tol * (tabs(sum) > big ? tabs(sum) : big)) break;
    prev = term;
  }
  return sum * ci;
}

// f_j (1/V) int lambda_j / X for one vertex j (sorted knots, any signs; PV across X = 0)
template <typename T> __device__ T inv_term_table(const T xin[4], const T f[4], int jj) {
  T x[4] = {xin[0], xin[1], xin[2], xin[3]};
  T s = tabs(x[0]) > tabs(x[3]) ? tabs(x[0]) : tabs(x[3]);
  if (s == T(0)) return T(0);
  const int nz = (x[0] == T(0)) + (x[1] == T(0)) + (x[2] == T(0)) + (x[3] == T(0));
  if (nz >= 3) {
#pragma unroll
    for (int l = 0; l < 4; ++l) x[l] = x[l] == T(0) ? T(kFloor) * s : x[l];
    T dummy[4] = {T(0), T(0), T(0), T(0)};
    sort4(x, dummy);
  }
  const T si = T(1) / s;
  T t5[5];
#pragma unroll
  for (int l = 0; l < 5; ++l) {
    const int src = l <= jj ? l : l - 1;
    t5[l] = (src == 0 ? x[0] : src == 1 ? x[1] : src == 2 ? x[2] : x[3]) * si;
  }
  const T fj = jj == 0 ? f[0] : jj == 1 ? f[1] : jj == 2 ? f[2] : f[3];
  return fj * dd5(t5) * si;
}

// sum_j f_j (1/V) int lambda_j / X for sorted knots x (any signs; PV across X = 0)
template <typename T> __device__ T inv_sum_table(const T xin[4], const T f[4]) {
  T x[4] = {xin[0], xin[1], xin[2], xin[3]};
  T s = tabs(x[0]) > tabs(x[3]) ? tabs(x[0]) : tabs(x[3]);
  if (s == T(0)) return T(0);
  const int nz = (x[0] == T(0)) + (x[1] == T(0)) + (x[2] == T(0)) + (x[3] == T(0));
  if (nz >= 3) {
    // a face with X = 0 (log-divergent): exact zeros floored, measure-zero input
#pragma unroll
    for (int l = 0; l < 4; ++l) x[l] = x[l] == T(0) ? T(kFloor) * s : x[l];
    // re-sort (floored zeros stay below the positive knots; negative knots stay first)
    T dummy[4] = {T(0), T(0), T(0), T(0)};
    sort4(x, dummy);
  }
  const T si = T(1) / s;
  T u[4];
#pragma unroll
  for (int l = 0; l < 4; ++l) u[l] = x[l] * si;
  T acc = T(0);
#pragma unroll 1
  for (int jj = 0; jj < 4; ++jj) {
    T t5[5];
    t5[0] = u[0];
#pragma unroll
    for (int l = 1; l < 5; ++l) t5[l] = l <= jj ? u[l] : u[l - 1];
    const T fj = jj == 0 ? f[0] : jj == 1 ? f[1] : jj == 2 ? f[2] : f[3];
    acc += fj * dd5(t5);
  }
  return acc * si;
}

// sum_j f_j (1/V) int lambda_j / X for sorted knots x (PV across X = 0) by one shared
// divided-difference table: with u = x/s (s = max|x|) and g(t) = t^3 ln|t|, the 4-knot entries
// G[p..r] are common to all j, and the entries with knot j doubled follow the same recursion,
//   H_j[p..r] = ((p < j ? H_j[p+1..r] : G[p..r]) - (r > j ? H_j[p..r-1] : G[p..r])) / (u_r - u_p),
//   H_j[j..j] = g'(u_j) = 3 u_j^2 ln|u_j| + u_j^2,
// so all four fourth divided differences g[u, u_j] = H_j[0..3] take four logarithms and six
// reciprocals (the per-vertex table below takes twenty and forty divisions).  The result is
// sum_j f_j H_j[0..3] / s.
// A pair of adjacent knots a < b of one sign with y = (b - a)/a small (|y| <= 1/8, ties
// included) would cancel in the recursion; its three entries g[a,b], g[a,a,b], g[a,b,b] are
// taken from the Taylor series about a instead (d = b - a):
//   g[a,b]   = g'(a) + d g2(a)/2 + d^2 g3(a)/6 + d sum_{k>=4} T_k
//   g[a,a,b] = g2(a)/2 + d g3(a)/6 + sum_{k>=4} T_k
//   g[a,b,b] = g2(a)/2 + d g3(a)/3 + sum_{k>=4} (k-1) T_k
// with the second and third derivatives g2 = 6t ln|t| + 5t, g3 = 6 ln|t| + 11, the higher ones
// 6 (-1)^k (k-4)!/a^(k-3) (k >= 4), and T_k = (k-th derivative at a) d^(k-2)/k! =
// 6 (-1)^k (k-4)!/k! a y^(k-2), which falls like y^k.  Two knots at 0 give the limits
// g'(0) = g''(0)/2 = 0.  Returns false, leaving the work to the per-vertex table, where two
// adjacent pairs both cluster (three knots together) or three knots are 0.
constexpr double kRhoShared = 0.125;  // adjacent knots this close (relative): series entries
template <typename T> __device__ __forceinline__ bool inv_sum_shared(const T x[4], const T f[4], T &out) {
  const T s = tabs(x[0]) > tabs(x[3]) ? tabs(x[0]) : tabs(x[3]);
  if (s == T(0)) {
    out = T(0);
    return true;
  }
  const T rho = T(kRhoShared);
  const T si = rcp(s);
  T u[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) u[i] = x[i] * si;
  int nz = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) nz += u[i] == T(0);
  if (nz >= 3) return false;
  bool cl[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const T a = u[i], b = u[i + 1];
    cl[i] = (a > T(0) && b - a <= rho * a) || (b < T(0) && b - a <= rho * (-b));
  }
  if ((cl[0] && cl[1]) || (cl[1] && cl[2])) return false;  // three knots together
  T g[4], gp[4], L[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const T t = u[i], t2 = t * t;
    L[i] = t == T(0) ? T(0) : Num<T>::lg(tabs(t));
    g[i] = t2 * t * L[i];
    gp[i] = T(3) * t2 * L[i] + t2;
  }
  // first-level entries of every adjacent pair: G1 = g[u_p, u_p+1], HL = g[u_p, u_p, u_p+1],
  // HR = g[u_p, u_p+1, u_p+1]
  T G1[3], HL[3], HR[3];
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const T d = u[p + 1] - u[p];
    if (!cl[p] && !(d > T(0))) {  // two knots at 0 (a tie elsewhere is clustered): the limits
      G1[p] = T(0);               // g'(0) = 0 and g''(0)/2 = 0
      HL[p] = T(0);
      HR[p] = T(0);
    } else if (!cl[p]) {
      const T r = rcp(d);
      G1[p] = (g[p + 1] - g[p]) * r;
      HL[p] = (G1[p] - gp[p]) * r;
      HR[p] = (gp[p + 1] - G1[p]) * r;
    } else {
      const T a = u[p], y = d * rcp(a), Lp = L[p];
      const T g2 = T(6) * a * Lp + T(5) * a, g3 = T(6) * Lp + T(11);
      // T_4 = a y^2 / 4; successive terms: T_{k+1} = -T_k (k-3) y / (k+1)
      T t = T(0.25) * a * y * y;
      T s0 = T(0), s1 = T(0);
#pragma unroll 1
      for (int k = 4; k < 4 + Num<T>::kmax; ++k) {
        s0 += t;
        s1 += T(k - 1) * t;
        if (tabs(t) <= Num<T>::tol * (tabs(s0) + tabs(g2) + tabs(g3))) break;
        t *= -T(k - 3) * y / T(k + 1);
      }
      HL[p] = T(0.5) * g2 + d * g3 * T(1.0 / 6.0) + s0;
      HR[p] = T(0.5) * g2 + d * g3 * T(1.0 / 3.0) + s1;
      G1[p] = gp[p] + d * (T(0.5) * g2 + d * g3 * T(1.0 / 6.0) + s0);
    }
  }
  const T r02 = rcp(u[2] - u[0]), r13 = rcp(u[3] - u[1]), r03 = rcp(u[3] - u[0]);
  const T G012 = (G1[1] - G1[0]) * r02, G123 = (G1[2] - G1[1]) * r13;
  const T G0123 = (G123 - G012) * r03;
  T R[4];
  {  // j = 0
    const T h02 = (G012 - HL[0]) * r02;
    R[0] = (G0123 - h02) * r03;
  }
  {  // j = 1
    const T h02 = (HL[1] - HR[0]) * r02, h13 = (G123 - HL[1]) * r13;
    R[1] = (h13 - h02) * r03;
  }
  {  // j = 2
    const T h02 = (HR[1] - G012) * r02, h13 = (HL[2] - HR[1]) * r13;
    R[2] = (h13 - h02) * r03;
  }
  {  // j = 3
    const T h13 = (HR[2] - G123) * r13;
    R[3] = (h13 - G0123) * r03;
  }
  out = (f[0] * R[0] + f[1] * R[1] + f[2] * R[2] + f[3] * R[3]) * si;
  return true;
}

// the shared table where it applies, else the per-vertex table
template <typename T> __device__ __forceinline__ T inv_sum_fast(const T x[4], const T f[4]) {
  T r;
  if (inv_sum_shared(x, f, r)) return r;
  return inv_sum_table(x, f);
}

// series branch: sorted knots of one sign with (x3 - x0) <= kappa |x0 + x3|
template <typename T> __device__ __forceinline__ bool series_ok(const T x[4], T kappa) {
  return (x[0] > T(0) || x[3] < T(0)) && (x[3] - x[0]) <= kappa * tabs(x[0] + x[3]);
}

// sum_j f_j (1/V) int_S lambda_j / X, sorted knots x (FP64 or FP32 throughout)
template <typename T> __device__ __forceinline__ T inv_sum(const T x[4], const T f[4]) {
  if (series_ok(x, T(Num<T>::kappa))) return series_sum(x, f);
  return inv_sum_fast(x, f);
}

// Mixed precision, knots of a final tetrahedron that missed the short series: the D = 0
// value of a vertex on both cut planes, interpolated in FP32 along different edges, comes
// out at the FP32 noise level of the corner energies instead of 0, so knots below 2^-20 of
// the largest are set to exactly 0 (the piece's integral moves by ~1e-5 relative; such
// pieces are a few in 10^4).  Returns true when the sorted knots keep an inner gap below
// tau times their scale (the near-degenerate case evaluated in FP64).
constexpr float kZeroSnap = 9.5367431640625e-07f;  // 2^-20
__device__ __forceinline__ bool mixed_knots(float x[4], const float d[4], float tau) {
  const float s = fmaxf(fabsf(d[0]), fabsf(d[3]));
#pragma unroll
  for (int i = 0; i < 4; ++i) x[i] = fabsf(d[i]) < kZeroSnap * s ? 0.0f : d[i];
  float g = s;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float gi = x[i + 1] - x[i];
    if (gi > 0.0f) g = fminf(g, gi);  // exact ties (e.g. two D = 0 vertices) are exact in FP32
  }
  return g < tau * s;
}

// FP32 evaluation of queued knots: the long series where it converges, else the table
__device__ __forceinline__ float inv_sum_long(const float x[4], const float f[4]) {
  if (series_ok(x, Num<float>::kappa_long)) return series_sum(x, f);
  return inv_sum_fast(x, f);
}

// mixed precision, all branches in one place (dynamic kernel)
__device__ __forceinline__ float inv_sum_mixed(const float d[4], const float f[4], float tau, int *fp64) {
  if (series_ok(d, Num<float>::kappa)) return series_sum(d, f);
  float x[4];
  if (!mixed_knots(x, d, tau)) return inv_sum_long(x, f);
  ++*fp64;
  double xd[4] = {x[0], x[1], x[2], x[3]}, fd[4] = {f[0], f[1], f[2], f[3]};
  return (float)inv_sum_table(xd, fd);
}

// Far-field moments of a final tetrahedron (sorted knots d >= 0, midpoint c > 0):
//   a_k = (-1)^k 6 k!/(k+4)! sum_j f_j h_k(e_1..e_4, e_j),  e = (d - c)/c,
// so that for any frequency w with rho = max|d - c| / |c - w| < 1
//   (1/V) sum_j f_j int_S lambda_j / (D - w) = (1/(c - w)) sum_k a_k z^k,  z = c / (c - w)
// (expansion of 1/(D - w) about c; at w = 0 this is the static series).  Writes a_0..a_{K-1}
// and returns K, the count after which |a_k| (times the largest z used, kappa c / max|d-c|)
// falls below tol.
template <typename T, int KMAX> __device__ int far_moments(const T d[4], const T f[4], T *a) {
  const T c = (d[0] + d[3]) * T(0.5);
  const T ci = rcp(c);
  T e[4];
#pragma unroll
  for (int l = 0; l < 4; ++l) e[l] = (d[l] - c) * ci;
  const T rmax = (d[3] - d[0]) * T(0.5) * ci;           // max|e|
  const T zmax = rmax > T(0) ? T(Num<T>::kappa_far) / rmax : T(1);  // largest |z| that uses them
  T H[4] = {T(1), T(1), T(1), T(1)};
  T P[4] = {T(1), T(1), T(1), T(1)};
  a[0] = T(0.25) * (f[0] + f[1] + f[2] + f[3]);
  const T ref = tabs(a[0]);
  T zk = T(1), prev = ref;
  int k = 1;
  for (; k < KMAX; ++k) {
    H[0] = e[0] * H[0];
#pragma unroll
    for (int l = 1; l < 4; ++l) H[l] = H[l - 1] + e[l] * H[l];
    T sj = T(0);
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      P[jj] = H[3] + e[jj] * P[jj];
      sj += f[jj] * P[jj];
    }
    a[k] = series_coef<T>(k) * sj;
    zk *= zmax;
    const T mag = tabs(a[k]) * zk;
    if (k >= 2 && mag + prev <= Num<T>::tol * ref) {
      ++k;
      break;
    }
    prev = mag;
  }
  return k;
}

// own-series terms for convergence ratio rho (rho^kk <= tol), at most K
template <typename T> __device__ __forceinline__ int own_terms(int K, T rho) {
  if (!(rho > T(0))) return K > 0 ? 1 : 0;
  const float need = __fdividef(Num<T>::log2_tol, __log2f((float)rho));  // rho^need = tol
  const int kk = 2 + (int)need;
  return kk < K ? kk : K;
}

// (1/(c - w)) sum_{k<kk} a_k z^k, z = c/(c - w), as two half-length Horner chains (even and
// odd powers: the weight kernels are bound by dependent latency); on the device, FP32
// coefficients are read in aligned pairs (a + k - 1 even: the caller's stride is even)
template <typename T> __device__ __forceinline__ T far_eval_k(const T *a, int kk, T c, T w) {
  const T den = c - w, rd = rcp(den);
  const T z = c * rd, z2 = z * z;
  T e = T(0), o = T(0);
  int k = kk - 1;
  if (k >= 0 && (k & 1) == 0) e = a[k--];
#pragma unroll 2
  for (; k >= 1; k -= 2) {
    T lo_, hi_;
#ifdef __CUDA_ARCH__
    if constexpr (sizeof(T) == 4) {
      const float2 pr = *reinterpret_cast<const float2 *>(a + k - 1);
      lo_ = pr.x;
      hi_ = pr.y;
    } else {
      lo_ = a[k - 1];
      hi_ = a[k];
    }
#else
    lo_ = a[k - 1];
    hi_ = a[k];
#endif
    o = o * z2 + hi_;
    e = e * z2 + lo_;
  }
  return (e + z * o) * rd;
}

// (1/(c - w)) sum_{k<K} a_k z^k with z = c/(c - w), truncated where rho^k < tol
template <typename T> __device__ __forceinline__ T far_eval(const T *a, int K, T c, T w, T rho) {
  return far_eval_k(a, own_terms(K, rho), c, w);
}

// Normalised cubic B-spline density M(w; t0..t4) (integral 1) by the de Boor-Cox
// recursion for M-splines; sorted knots, half-open support.
template <typename T> __device__ __forceinline__ T mspline5(const T t[5], T w) {
  T M[4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
    M[i] = (t[i] <= w && w < t[i + 1]) ? T(1) / (t[i + 1] - t[i]) : T(0);
#pragma unroll
  for (int k = 2; k <= 4; ++k) {
#pragma unroll
    for (int i = 0; i + k <= 4; ++i) {
      const T den = t[i + k] - t[i];
      M[i] = den > T(0) ? T(k) * ((w - t[i]) * M[i] + (t[i + k] - w) * M[i + 1]) / (T(k - 1) * den)
                        : T(0);
    }
  }
  return M[0];
}

// sum_j f_j (1/V) int_S lambda_j delta(w - D) = (1/4) sum_j f_j M(w; d, d_j), sorted d
template <typename T> __device__ __forceinline__ T delta_sum(const T d[4], const T f[4], T w) {
  if (!(w > d[0] && w < d[3])) return T(0);
  T acc = T(0);
#pragma unroll
  for (int jj = 0; jj < 4; ++jj) {
    T t5[5];
#pragma unroll
    for (int l = 0; l < 5; ++l) t5[l] = l <= jj ? d[l] : d[l - 1];
    acc += f[jj] * mspline5(t5, w);
  }
  return T(0.25) * acc;
}

// delta_sum at w = 0 for knots x already shifted by the frequency, with the reciprocals rs of the
// knot spans 01, 12, 23, 02, 13, 03 given (they do not depend on the shift): the same de Boor-Cox
// recursion per vertex, multiplying by the reciprocal spans instead of dividing.  (The B-spline
// recursion combines nonnegative terms, so spans from the unshifted knots cost no accuracy; the
// divided-difference table of the principal value keeps the differences of its own rounded knots.)
template <typename T> __device__ __forceinline__ T delta_sum_pre(const T x[4], const T f[4], const T rs[6]) {
  if (!(x[0] < T(0) && x[3] > T(0))) return T(0);
  // reciprocal span of original knots a <= b (0 for a == b)
  auto R = [&](int a, int b) -> T {
    if (a == b) return T(0);
    const int k = b - a;
    return k == 1 ? rs[a] : (k == 2 ? rs[3 + a] : rs[5]);
  };
  T acc = T(0);
#pragma unroll
  for (int jj = 0; jj < 4; ++jj) {
    int id[5];
    T t[5];
#pragma unroll
    for (int l = 0; l < 5; ++l) {
      id[l] = l <= jj ? l : l - 1;
      t[l] = x[id[l]];
    }
    T M[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) M[i] = (t[i] <= T(0) && T(0) < t[i + 1]) ? R(id[i], id[i + 1]) : T(0);
#pragma unroll
    for (int k = 2; k <= 4; ++k) {
#pragma unroll
      for (int i = 0; i + k <= 4; ++i) {
        const T den = t[i + k] - t[i];
        M[i] = den > T(0) ? (T(k) / T(k - 1)) * ((-t[i]) * M[i] + t[i + k] * M[i + 1]) * R(id[i], id[i + k]) : T(0);
      }
    }
    acc += f[jj] * M[0];
  }
  return T(0.25) * acc;
}

// Tetrahedron density of states at eF for one band: M(0; a_0..a_3), quadratic B-spline
template <typename T> __device__ __forceinline__ T dos4(T a0, T a1, T a2, T a3) {
  T t[4] = {a0, a1, a2, a3};
  T dm[4] = {T(0), T(0), T(0), T(0)};
  sort4(t, dm);
  if (!(T(0) >= t[0] && T(0) < t[3])) return T(0);
  T M[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) M[i] = (t[i] <= T(0) && T(0) < t[i + 1]) ? T(1) / (t[i + 1] - t[i]) : T(0);
#pragma unroll
  for (int k = 2; k <= 3; ++k) {
#pragma unroll
    for (int i = 0; i + k <= 3; ++i) {
      const T den = t[i + k] - t[i];
      M[i] = den > T(0) ? T(k) * ((T(0) - t[i]) * M[i] + (t[i + k] - T(0)) * M[i + 1]) /
                              (T(k - 1) * den)
                        : T(0);
    }
  }
  return M[0];
}

// ------------------------------------------------------------------------------------
// carving (Sec. II, Fig. 1): keep the part of a tetrahedron where the key is negative.
// WHICH = 0: key = a (first carving, occupied states); WHICH = 1: key = -b (second
// carving, empty states at k+q).  Each piece is emitted with its volume relative to the
// cut tetrahedron, from the cut fractions along the edges.
// ------------------------------------------------------------------------------------
// vertex: a = e^m_k - eF, D = e^n_{k+q} - e^m_k (b = a + D), f = |M|^2; D is its own
// linear attribute so it is exactly 0 wherever the corner data make it 0
template <typename T> struct Vt {
  T a, D, f;
};

template <typename T> __device__ __forceinline__ Vt<T> vmix(const Vt<T> &P, const Vt<T> &Q, T t) {
  const T s = T(1) - t;
  return Vt<T>{s * P.a + t * Q.a, s * P.D + t * Q.D, s * P.f + t * Q.f};
}

template <int WHICH, typename T> __device__ __forceinline__ T vkey(const Vt<T> &v) {
  return WHICH == 0 ? v.a : -(v.a + v.D);
}

// point where the key vanishes on edge P (key < 0) - Q (key >= 0); returns the fraction
template <int WHICH, typename T>
__device__ __forceinline__ Vt<T> vcut(const Vt<T> &P, const Vt<T> &Q, T &frac) {
  const T kp = vkey<WHICH>(P), kq = vkey<WHICH>(Q);
  frac = quot(kp, kp - kq);
  Vt<T> R = vmix(P, Q, frac);
  if (WHICH == 0) R.a = T(0);  // on the first cut plane; the second cut is the last one
  return R;
}

template <int WHICH, typename T> __device__ __forceinline__ void vswap(Vt<T> &x, Vt<T> &y) {
  if (vkey<WHICH>(y) < vkey<WHICH>(x)) {
    Vt<T> t = x; x = y; y = t;
  }
}

// Piece idx of one cut (keep key < 0) and the number of pieces (0, 1 or 3); r = volume of
// the piece relative to the input tetrahedron, from the cut fractions along the edges.
// Pieces are built on demand so that only one of them is live at a time.
template <int WHICH, typename T>
__device__ __forceinline__ int cut_piece(const Vt<T> in[4], int idx, Vt<T> P[4], T &r) {
  Vt<T> S[4] = {in[0], in[1], in[2], in[3]};
  vswap<WHICH>(S[0], S[1]);
  vswap<WHICH>(S[2], S[3]);
  vswap<WHICH>(S[0], S[2]);
  vswap<WHICH>(S[1], S[3]);
  vswap<WHICH>(S[1], S[2]);
  const int nneg = (vkey<WHICH>(S[0]) < T(0)) + (vkey<WHICH>(S[1]) < T(0)) +
                   (vkey<WHICH>(S[2]) < T(0)) + (vkey<WHICH>(S[3]) < T(0));
  if (nneg == 0) return 0;
  if (nneg == 4) {
#pragma unroll
    for (int i = 0; i < 4; ++i) P[i] = S[i];
    r = T(1);
    return 1;
  }
  if (nneg == 1) {  // corner tetrahedron at S0: volume t1 t2 t3
    T t1, t2, t3;
    P[0] = S[0];
    P[1] = vcut<WHICH>(S[0], S[1], t1);
    P[2] = vcut<WHICH>(S[0], S[2], t2);
    P[3] = vcut<WHICH>(S[0], S[3], t3);
    r = t1 * t2 * t3;
    return 1;
  }
  if (nneg == 2) {  // prism (S0, P02, P03) - (S1, P12, P13)
    T u0, v0, u1, v1;
    const Vt<T> P02 = vcut<WHICH>(S[0], S[2], u0), P03 = vcut<WHICH>(S[0], S[3], v0);
    const Vt<T> P12 = vcut<WHICH>(S[1], S[2], u1), P13 = vcut<WHICH>(S[1], S[3], v1);
    if (idx == 0) {
      P[0] = S[0]; P[1] = P02; P[2] = P03; P[3] = S[1];
      r = u0 * v0;
    } else if (idx == 1) {
      P[0] = P02; P[1] = P03; P[2] = S[1]; P[3] = P12;
      r = v0 * (T(1) - u0) * u1;
    } else {
      P[0] = P03; P[1] = S[1]; P[2] = P12; P[3] = P13;
      r = (T(1) - v0) * u1 * v1;
    }
    return 3;
  }
  // nneg == 3: tetrahedron minus the corner at S3: prism (S0,S1,S2) - (P03,P13,P23)
  T s0, s1, s2;
  const Vt<T> P03 = vcut<WHICH>(S[0], S[3], s0), P13 = vcut<WHICH>(S[1], S[3], s1),
              P23 = vcut<WHICH>(S[2], S[3], s2);
  if (idx == 0) {
    P[0] = S[0]; P[1] = S[1]; P[2] = S[2]; P[3] = P03;
    r = s0;
  } else if (idx == 1) {
    P[0] = S[1]; P[1] = S[2]; P[2] = P03; P[3] = P13;
    r = (T(1) - s0) * s1;
  } else {
    P[0] = S[2]; P[1] = P03; P[2] = P13; P[3] = P23;
    r = (T(1) - s0) * (T(1) - s1) * s2;
  }
  return 3;
}

// Both carvings of one (tetrahedron, band pair): emit(vol_ratio, d[4], f[4]) for every
// final tetrahedron (d = b - a >= 0, unsorted).  Rolled loops: one copy of the emitted
// body, one live piece per level.
template <typename T, typename Emit>
__device__ __forceinline__ void carve2(const T a[4], const T b[4], const T f[4], Emit &&emit) {
  const T amax = fmax(fmax(a[0], a[1]), fmax(a[2], a[3]));
  const T bmin = fmin(fmin(b[0], b[1]), fmin(b[2], b[3]));
  if (amax < T(0) && bmin > T(0)) {  // occupied at k and empty at k+q everywhere: no cut
    T d[4] = {b[0] - a[0], b[1] - a[1], b[2] - a[2], b[3] - a[3]};
    T ff[4] = {f[0], f[1], f[2], f[3]};
    emit(T(1), d, ff);
    return;
  }
  Vt<T> V[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) V[i] = Vt<T>{a[i], b[i] - a[i], f[i]};
#pragma unroll 1
  for (int i1 = 0; i1 < 3; ++i1) {
    Vt<T> P[4];
    T r1 = T(0);
    const int n1 = cut_piece<0>(V, i1, P, r1);
    if (i1 >= n1) break;
    if (r1 <= T(0)) continue;
#pragma unroll 1
    for (int i2 = 0; i2 < 3; ++i2) {
      Vt<T> Qv[4];
      T r2 = T(0);
      const int n2 = cut_piece<1>(P, i2, Qv, r2);
      if (i2 >= n2) break;
      const T r = r1 * r2;
      if (r <= T(0)) continue;
      T d[4], ff[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const T dd = Qv[i].D;
        d[i] = dd > T(0) ? dd : T(0);
        ff[i] = Qv[i].f;
      }
      emit(r, d, ff);
    }
  }
}


// Carving with the D attribute as an offset: every vertex carries e = D - D0 for one
// reference value D0 per band pair (passed as koff = D0 rounded to T), so that knots near a
// frequency w can be formed as (D0 - w) + e without the rounding of D0 itself (the
// dynamic kernel's mixed path).  First cut on a, second on b = a + koff + e; the emitted
// pieces carry offsets e (clamped to D >= 0).
template <typename T, typename Emit>
__device__ __forceinline__ void carve2_off(const T a[4], const T e[4], T koff, const T f[4], Emit &&emit) {
  const T amax = fmax(fmax(a[0], a[1]), fmax(a[2], a[3]));
  const T bmin = fmin(fmin(a[0] + koff + e[0], a[1] + koff + e[1]), fmin(a[2] + koff + e[2], a[3] + koff + e[3]));
  if (amax < T(0) && bmin > T(0)) {
    T ee[4] = {e[0], e[1], e[2], e[3]};
    T ff[4] = {f[0], f[1], f[2], f[3]};
    emit(T(1), ee, ff);
    return;
  }
  Vt<T> V[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) V[i] = Vt<T>{a[i], e[i], f[i]};
#pragma unroll 1
  for (int i1 = 0; i1 < 3; ++i1) {
    Vt<T> P[4];
    T r1 = T(0);
    const int n1 = cut_piece<0>(V, i1, P, r1);
    if (i1 >= n1) break;
    if (r1 <= T(0)) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) P[i].a += koff;  // second-cut key -(a + e) is now -b
#pragma unroll 1
    for (int i2 = 0; i2 < 3; ++i2) {
      Vt<T> Qv[4];
      T r2 = T(0);
      const int n2 = cut_piece<1>(P, i2, Qv, r2);
      if (i2 >= n2) break;
      const T r = r1 * r2;
      if (r <= T(0)) continue;
      T ee[4], ff[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        ee[i] = Qv[i].D > -koff ? Qv[i].D : -koff;
        ff[i] = Qv[i].f;
      }
      emit(r, ee, ff);
    }
  }
}

// x - y = s + t exactly (Knuth's two-difference; any order of magnitudes)
__device__ __forceinline__ void two_diff(float x, float y, float &s, float &t) {
  s = x - y;
  const float bb = s - x;
  t = (x - (s - bb)) - (y + bb);
}

}  // namespace chi0dev
