// chi0_dynamic.cu -- frequency-resolved weights of the doubly carved tetrahedron method:
// Re chi0 as the principal value of Eq. 1, Im chi0 from the delta function of Eq. 2, odd in w
// (Eq. 3), on every final tetrahedron of the two carvings of Sec. II, for one pass of up to
// 256 frequencies.
//
// Per final tetrahedron S (knots d_j of D, values f_j of |M|^2, weight v = volume fraction):
//   Re(u) += v sum_j f_j (1/V) int_S lambda_j [1/(D - u) + 1/(D + u)],   u = |w|
//   Im(w) += sign(w) pi v sum_j f_j (1/V) int_S lambda_j delta(u - D)
// The delta term is nonzero only for u inside (d_0, d_3) and is always evaluated piece by
// piece.  The principal-value terms are smooth in u away from the knots, so for frequencies
// far from a piece they are gathered per box of D instead of per (piece, frequency):
//
//   box b: centre C_b, radius R_b; every piece assigned to it has |d_j - C_b| <= R_b, and adds
//     its moments  M_k += v sum_j f_j (1/V) int_S lambda_j eps^k,  eps = (D - C_b)/R_b,
//     = v 6 k!/(k+4)! sum_j f_j h_k(e_1..e_4, e_j)  (e = (d - C_b)/R_b; Dirichlet moments of
//     the simplex, h_k the complete homogeneous symmetric polynomials);
//   1/(D -+ u) = 1/(C_b -+ u) sum_k (-z)^k eps^k,  z = R_b/(C_b -+ u),  |z| <= 1/2 where the
//     box stands in for its pieces (1/3 in FP64), so the box's share of Re(u) is
//     sum_k M_k (-z)^k/(C_b -+ u),
//     evaluated once per (box, frequency) in FP64 after the moments of all warps are summed.
//
// Boxes (rebuilt each pass from u_max = max |w| of the pass):
//   fine boxes, levels l = 0..3 of width w_l = (u_max/32) 2^l: centres (j + 1/2) w_l, radius
//     w_l; a piece of half-width s <= w_l/2 whose centre lies in [j w_l, (j+1) w_l) fits.  For a
//     frequency with |C_b - u| < F R_b (the - term) or C_b + u < F R_b (the + term), F = 2 in
//     the FP32 kernel and 3 in the FP64 kernel (|z| <= 1/F elsewhere), the box does not stand
//     in: its pieces evaluate that term themselves (own far-field series about their midpoint,
//     or the divided-difference table near their knots);
//   geometric boxes past u_max: x = c - u_max in [x_b, 1.25 x_b), x_0 = 5 u_max/32, centre
//     u_max + 1.125 x_b, radius x_b/4, pieces with s <= x_b/8; every frequency of the pass is
//     far (|z| <= 2/9), so their pieces evaluate nothing per frequency;
//   pieces wider than any box, or past the last one, are evaluated at every frequency.
// Every (piece, frequency, term) is taken exactly once, either by the piece or by its box;
// the predicate that decides is computed in the kernels' precision from the same table.
//
// Work layout.  A warp takes a batch of 32 tetrahedra; the batch's (m, n) items are sorted
// into whole-tetrahedron and cut lists and carved 32 at a time, one item per lane, in warp-
// uniform steps that emit at most one final tetrahedron per lane.  Each piece finds its box
// and moments in its lane (one lane per moment index adds them to the box sums).  Pieces that
// evaluate frequencies themselves (fine boxes, or no box) go to a per-warp ring queue that the
// whole warp drains 32 pieces at a time: own series with lanes owning frequencies, then the
// near-field (piece, frequency, term) entries of all of them packed one per lane; entries the
// shared divided-difference table leaves go to a per-warp fallback buffer in global memory,
// evaluated in full rounds when it fills.
// Sums.  FP32 kernel: per-CTA sums in 64-bit fixed point (units of 2^-44) in shared memory,
// added with integer atomics and written once per CTA: integer sums are exact in any order, so
// the warps take batches from a launch-wide counter (balanced loads) and the results are
// bitwise reproducible for any launch shape.  FP64 kernel: per-warp compensated FP64 sums per
// batch, batches assigned statically (batch = warp + k * warps), every sum in a fixed order:
// bitwise reproducible for a given launch shape.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "chi0_grid.cuh"
#include "chi0_internal.h"
#include "chi0_math.cuh"

using namespace chi0dev;

namespace chi0int {
namespace {

using grid::div_small;
using grid::kFull;
using grid::tet_corners;

constexpr int kNWPass = 256;   // frequencies per dynamic pass
// FP32 kernel: sums in 64-bit fixed point, units of 2^-44 (exact and order-independent; every
// per-CTA total stays far below 2^19, and one rounding of 2^-45 per term is far below the
// FP32 terms' own error)
constexpr float kFxScale = 17592186044416.0f;  // 2^44
constexpr double kFxUnit = 1.0 / 17592186044416.0;
constexpr int kNearCap = 1024;  // near-field (piece, frequency, term) entries listed per warp
constexpr int kFbCap = 4096;   // near-field entries left to the per-vertex table, per warp
static_assert(kFbCap >= 4 * kNearCap, "the fallback buffer holds several near lists' leftovers");
static_assert(kNearCap >= 4 * kNWPass, "the near list keeps room for two pieces' entries");

// a near-field entry the shared table leaves: knots x (sorted), values f, weight v, and
// code = frequency index << 2 | term << 1 | (w < 0)
template <typename T> struct FbEnt {
  T x[4], f[4], v;
  int code;
};

template <bool FP64> struct DynShape {
  static constexpr int threads = FP64 ? 64 : 128;
  static constexpr int warps = threads / 32;
  static constexpr int DC = FP64 ? 16 : 32;  // queued pieces evaluated per round
  static constexpr int KM = FP64 ? 64 : 32;  // own far-field moments kept per queued piece
  static constexpr int NF = FP64 ? 3 : 2;    // a fine box stands in beyond NF radii
  static constexpr int KF = FP64 ? 28 : 24;  // moments of a fine box   (truncation NF^-KF)
  static constexpr int KG = FP64 ? 22 : 12;  // moments of a geometric box ((2/9)^KG)
};

// box geometry
constexpr int kBoxL = 4;      // fine levels
constexpr int kBoxJ0 = 32;    // finest boxes across [0, u_max]
constexpr int kBoxExtra = 6;  // fine boxes per level past u_max
constexpr int kBoxG = 40;     // geometric boxes (x_0 1.25^40 = 7500 x_0)
constexpr int kMinBoxNw = 8;  // fewer frequencies: every piece evaluates all of them
__host__ __device__ constexpr int box_J(int l) { return (kBoxJ0 >> l) + kBoxExtra; }
constexpr int kBoxFine = box_J(0) + box_J(1) + box_J(2) + box_J(3);
constexpr int kBoxes = kBoxFine + kBoxG;
template <bool FP64> __host__ __device__ constexpr int box_slots() {
  return kBoxFine * DynShape<FP64>::KF + kBoxG * DynShape<FP64>::KG;
}
template <bool FP64> __host__ __device__ constexpr int slot_base(int b) {
  return b < kBoxFine ? b * DynShape<FP64>::KF
                      : kBoxFine * DynShape<FP64>::KF + (b - kBoxFine) * DynShape<FP64>::KG;
}

// the pass's boxes in the kernels' precision (written by k_box_setup, read by both kernels)
template <typename T> struct BoxTab {
  T C[kBoxes], R[kBoxes];  // centre and radius
  T lowG[kBoxG + 1];       // lower edges x_b of the geometric boxes (x = c - u_max)
  T W0, x0, umax;
  int on;
};

template <typename T> __device__ __forceinline__ void kadd_t(T &sum, T &comp, T x) {
  const T t = sum + x;
  if (tabs(sum) >= tabs(x)) comp += (sum - t) + x;
  else comp += (x - t) + sum;
  sum = t;
}

// one block: u_max of the pass and the box table
template <typename T>
__global__ void __launch_bounds__(256) k_box_setup(const double *__restrict__ omega, int nw, BoxTab<T> *tab) {
  __shared__ double red[8];
  double u = 0.0;
  for (int i = threadIdx.x; i < nw; i += blockDim.x) u = fmax(u, fabs(omega[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) u = fmax(u, __shfl_xor_sync(kFull, u, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = u;
  __syncthreads();
  double umax = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) umax = fmax(umax, red[i]);
  const T W0 = (T)(umax / kBoxJ0), um = (T)umax, x0 = W0 * T(5);
  const int on = (nw >= kMinBoxNw && umax > 1e-30 && umax < 1e30 && W0 > T(0)) ? 1 : 0;
  if (threadIdx.x == 0) {
    tab->W0 = W0;
    tab->x0 = x0;
    tab->umax = um;
    tab->on = on;
    double lo = (double)x0;
    for (int b = 0; b <= kBoxG; ++b) {
      tab->lowG[b] = (T)lo;
      lo *= 1.25;
    }
  }
  __syncthreads();
  const int b = threadIdx.x;
  if (b < kBoxFine) {
    int l = 0, j = b;
    while (j >= box_J(l)) {
      j -= box_J(l);
      ++l;
    }
    const T w = W0 * (T)(1 << l);
    tab->C[b] = ((T)j + T(0.5)) * w;
    tab->R[b] = w;
  } else if (b < kBoxes) {
    const T xb = tab->lowG[b - kBoxFine];
    tab->C[b] = um + xb * T(1.125);
    tab->R[b] = xb * T(0.25);
  }
}

// box of a final tetrahedron with midpoint c and half-width s (-1: none, evaluate directly)
template <typename T> __device__ __forceinline__ int box_of(T c, T s, const BoxTab<T> &tb) {
  if (!tb.on) return -1;
  const T x = c - tb.umax;
  if (x >= tb.x0) {
    int b = (int)(__log2f((float)quot(x, tb.x0)) * 3.1062837f);  // log base 1.25 (a first guess)
    b = b < 0 ? 0 : (b > kBoxG - 1 ? kBoxG - 1 : b);
    while (b > 0 && x < tb.lowG[b]) --b;
    while (b < kBoxG - 1 && x >= tb.lowG[b + 1]) ++b;
    if (x >= tb.lowG[b] && x < tb.lowG[b + 1] && s <= T(0.125) * tb.lowG[b]) return kBoxFine + b;
  }
  T w = tb.W0;
  int off = 0;
#pragma unroll 1
  for (int l = 0; l < kBoxL; ++l) {
    if (s <= T(0.5) * w) {
      const T jf = floor(quot(c, w));
      return jf < (T)box_J(l) ? off + (int)jf : -1;
    }
    off += box_J(l);
    w *= T(2);
  }
  return -1;
}

// moments m_k = v 6 k!/(k+4)! sum_j f_j h_k(e, e_j), k < K, of a piece about a box (e = (d - C)/R)
template <typename T> __device__ __noinline__ void box_moments_ol(const T e[4], const T f[4], T v, T *m, int K) {
  T H[4] = {T(1), T(1), T(1), T(1)};
  T P[4] = {T(1), T(1), T(1), T(1)};
  m[0] = v * T(0.25) * (f[0] + f[1] + f[2] + f[3]);
  for (int k = 1; k < K; ++k) {
    H[0] = e[0] * H[0];
#pragma unroll
    for (int l = 1; l < 4; ++l) H[l] = H[l - 1] + e[l] * H[l];
    T sj = T(0);
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      P[jj] = H[3] + e[jj] * P[jj];
      sj += f[jj] * P[jj];
    }
    m[k] = v * tabs(series_coef<T>(k)) * sj;
  }
}

// the same moments added straight into fixed-point box sums dst[0..K) (shared-memory atomics)
__device__ __forceinline__ void box_moments_fx(const float e[4], const float f[4], float v, unsigned long long *dst,
                                               int K) {
  float H[4] = {1.f, 1.f, 1.f, 1.f};
  float P[4] = {1.f, 1.f, 1.f, 1.f};
  // (terms that round to 0 in fixed point are skipped: high moments of small pieces)
  long long t0 = __float2ll_rn(v * 0.25f * (f[0] + f[1] + f[2] + f[3]) * kFxScale);
  if (t0) atomicAdd(&dst[0], (unsigned long long)t0);
#pragma unroll 1
  for (int k = 1; k < K; ++k) {
    H[0] = e[0] * H[0];
#pragma unroll
    for (int l = 1; l < 4; ++l) H[l] = H[l - 1] + e[l] * H[l];
    float sj = 0.f;
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      P[jj] = H[3] + e[jj] * P[jj];
      sj += f[jj] * P[jj];
    }
    const long long t = __float2ll_rn(v * tabs(series_coef<float>(k)) * sj * kFxScale);
    if (t) atomicAdd(&dst[k], (unsigned long long)t);
  }
}

// Out-of-line copy of the fallback's delta term: inlined copies of the helpers at several call
// sites made the kernel's body overflow the instruction cache (ncu: 45% of the issue stalls
// waiting for instructions).  Helpers with one call site (the near drain's divided-difference
// table and de Boor recursion, the own and the box moments) are inlined there: 8% and 3%
// faster than calling them.
template <typename T> __device__ __noinline__ T delta_sum_ol(const T d[4], const T f[4]) { return delta_sum(d, f, T(0)); }

// does box b stand in for term (0: 1/(D - u), 1: 1/(D + u)) at frequency u = om?  Fine boxes
// only near themselves; geometric boxes always.  Same expression in both kernels.
template <typename T> __device__ __forceinline__ bool box_far(T C, T R, int b, T om, int term) {
  if (b >= kBoxFine) return true;
  const T r2 = R * T(DynShape<sizeof(T) == 8>::NF);
  if (term) return !(C + om < r2);
  return !(tabs(C - om) < r2);
}

// sum_j f_j (1/V) int lambda_j / X for knots x of X near 0: divided-difference table (principal
// value across X = 0); one out-of-line copy shared by every call site
template <bool FP64>
__device__ __noinline__ typename std::conditional<FP64, double, float>::type near_term(
    const typename std::conditional<FP64, double, float>::type *x,
    const typename std::conditional<FP64, double, float>::type *f, float tau, int &nfp64) {
  using T = typename std::conditional<FP64, double, float>::type;
  T xx[4] = {x[0], x[1], x[2], x[3]};
  // (the entries that reach this function are the ones the shared table left: the per-vertex
  // table directly, after the series branches)
  if constexpr (FP64) {
    if (series_ok(xx, T(Num<T>::kappa))) return series_sum(xx, f);
    return inv_sum_table(xx, f);
  } else {
    if (series_ok(xx, Num<float>::kappa)) return series_sum(xx, f);
    float y[4];
    if (!mixed_knots(y, xx, tau)) {
      if (series_ok(y, Num<float>::kappa_long)) return series_sum(y, f);
      return inv_sum_table(y, f);
    }
    ++nfp64;
    double yd[4] = {y[0], y[1], y[2], y[3]}, fd[4] = {f[0], f[1], f[2], f[3]};
    return (float)inv_sum_table(yd, fd);
  }
}

// D0 - w for a frequency near the knots: with D0 = D0h + D0l and w = wh + wl split into
// FP32 parts the difference keeps full relative precision however close D0 is to w
__device__ __forceinline__ float near_shift(float D0h, float D0l, float wh, float wl) {
  float sv, tv;
  two_diff(D0h, wh, sv, tv);
  return sv + (tv + (D0l - wl));
}
__device__ __forceinline__ double near_shift(double D0h, double, double wh, double) { return D0h - wh; }

// knots of near-field entry ent (= 2 * frequency index + term) of a piece with knots
// d = D0 + e (sorted), D0 = D0h + D0l: term 0 is 1/(D - |w|) with knots (D0 - |w|) + e, term 1
// is 1/(D + |w|) with knots d + |w|
template <bool FP64, typename T>
__device__ __forceinline__ void near_knots(int ent, const T d[4], const T e[4], T D0h, T D0l, const T *s_w,
                                           const T *s_wl, T x[4], bool &neg) {
  const int iw = ent >> 1, sgn = ent & 1;
  const T w = s_w[iw];
  neg = w < T(0);
  const T om = neg ? -w : w;
  if (sgn) {
#pragma unroll
    for (int i = 0; i < 4; ++i) x[i] = d[i] + om;
  } else {
    const T sh = near_shift(D0h, D0l, om, FP64 ? T(0) : (neg ? -s_wl[iw] : s_wl[iw]));
#pragma unroll
    for (int i = 0; i < 4; ++i) x[i] = sh + e[i];
  }
}

// IMO: Im only (the delta term of Eq. 2 on an ascending grid of w >= 0; no principal value,
// no boxes) for the Kramers-Kronig route to Re
template <bool FP64, bool IMO = false>
__global__ void __launch_bounds__(DynShape<FP64>::threads, FP64 ? 2 : 3)
    k_dynamic(Grid g, Tet tet, const void *__restrict__ Ek, const void *__restrict__ Ekq, Q q,
              const void *__restrict__ W2, int cma, float tau, const short *__restrict__ occ,
              const short *__restrict__ empq, const double *__restrict__ omega, int nw, DynBufs db,
              const float *__restrict__ Eklo, const float *__restrict__ Ekqlo,
              unsigned long long *__restrict__ counters) {
  using T = typename std::conditional<FP64, double, float>::type;
  using S = DynShape<FP64>;
  constexpr int W = S::warps, KM = S::KM, KF = S::KF, KG = S::KG, DC = S::DC;
  constexpr int QC = 64;  // queue of final tetrahedra that evaluate frequencies themselves
  constexpr int NS = box_slots<FP64>();
  // per-piece strides of the scratch: odd (conflict-free lane-parallel writes), except the FP32
  // own moments, even so that the own series reads them in aligned pairs (2-way write conflicts)
  constexpr int SKM = FP64 ? KM + 1 : KM + 2, SKF = KF + 1;
  constexpr int KU = DC * SKM > 32 * SKF ? DC * SKM : 32 * SKF;  // per-warp scratch (T elements)
  static_assert(QC >= DC + 32, "one carving step adds at most 32 queued pieces");
  __shared__ int s_c[W][32][4], s_cq[W][32][4];
  __shared__ T s_vol[W][32];
  __shared__ int s_nlo[W][32], s_nn[W][32], s_pre[W][33];
  __shared__ int s_list[W][2][64], s_nl[W][2];  // item lists (whole / cut): l << 24 | m << 12 | n
  // scratch: box moments of one carving step's pieces (32 x KF), or the own far-field moments
  // of the queued pieces being evaluated (DC x KM)
  __shared__ T s_scr[W][KU];
  __shared__ int s_pk[W][DC];
  // ring queue: offsets e from D0 (sorted), values f, (weight, D0h, D0l), box
  __shared__ __align__(16) T s_qe[W][QC][4];
  __shared__ __align__(16) T s_qf[W][QC][4];
  __shared__ T s_qv[W][QC][3];
  __shared__ int s_qb[W][QC];
  // FP64 kernel: per-warp compensated sums of the batch (static batch order); FP32 kernel:
  // per-CTA fixed-point sums of the whole launch (s_fx; batches in any order)
  constexpr bool FX = !FP64;
  constexpr int WA = FX ? 1 : W, NA = FX ? 1 : kNWPass;
  __shared__ T sR[WA][NA], sI[WA][NA];
  __shared__ T cR[WA][NA], cI[WA][NA];  // compensation terms
  __shared__ unsigned long long s_fx[FX ? 2 : 1][FX ? kNWPass : 1];
  __shared__ T s_w[kNWPass];
  __shared__ T s_wl[FP64 ? 1 : kNWPass];  // FP32 path: w - (float)w
  // near-field entries of the drain's pieces: ring slot << 9 | 2 * frequency index + term
  __shared__ unsigned short s_near[W][kNearCap];
  __shared__ short s_rng[kBoxFine][2];  // frequencies a fine box leaves to its pieces: [lo, hi)
  __shared__ BoxTab<T> s_tab;
  extern __shared__ __align__(16) unsigned char s_dyn[];  // box sums: [W][NS] (FP64), [NS] fixed point
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  T *acc = (T *)s_dyn + (size_t)wib * NS;
  unsigned long long *bfx = (unsigned long long *)s_dyn;
  T *scr = s_scr[wib];
  const int w = q.hi - q.lo;
  const long long nbatch = (g.ntet + 31) / 32;
  const long long gwarp = (long long)blockIdx.x * W + wib, nwarps = (long long)gridDim.x * W;
  double *gpart = db.box_part + gwarp * NS;
  FbEnt<T> *gfb = (FbEnt<T> *)db.fb + gwarp * kFbCap;
#pragma unroll 1
  for (int iw = threadIdx.x; iw < nw; iw += blockDim.x) {
    s_w[iw] = (T)omega[iw];
    if constexpr (!FP64) s_wl[iw] = (float)(omega[iw] - (double)s_w[iw]);
  }
  {
    if constexpr (IMO) {
      if (threadIdx.x == 0) s_tab.on = 0;  // every piece evaluates its own frequencies
    } else {
      const BoxTab<T> *src = (const BoxTab<T> *)db.box_tab;
      const int nwords = (int)(sizeof(BoxTab<T>) / 4);
#pragma unroll 1
      for (int i = threadIdx.x; i < nwords; i += blockDim.x) ((int *)&s_tab)[i] = ((const int *)src)[i];
    }
  }
  if constexpr (FX) {
    if constexpr (!IMO) {
#pragma unroll 1
      for (int i = threadIdx.x; i < NS; i += blockDim.x) bfx[i] = 0ull;
    }
#pragma unroll 1
    for (int i = threadIdx.x; i < 2 * kNWPass; i += blockDim.x) s_fx[i / kNWPass][i % kNWPass] = 0ull;
  } else {
#pragma unroll 1
    for (int i = lane; i < (IMO ? 0 : NS); i += 32) acc[i] = T(0);
  }
  __syncthreads();
  // frequency ranges of the fine boxes: contiguous when |w| ascends along the grid (an
  // interval for the - term, a prefix for the + term); otherwise the whole grid, the
  // predicate deciding each frequency
  bool sorted = true;
#pragma unroll 1
  for (int i = threadIdx.x; i + 1 < nw; i += blockDim.x) sorted = sorted && tabs(s_w[i]) <= tabs(s_w[i + 1]);
  sorted = __syncthreads_and(sorted) != 0;
#pragma unroll 1
  for (int b = threadIdx.x; b < (IMO ? 0 : kBoxFine); b += blockDim.x) {
    int lo = 0, hi = nw;
    if (sorted) {
      lo = nw;
      hi = 0;
#pragma unroll 1
      for (int i = 0; i < nw; ++i) {
        const T om = tabs(s_w[i]);
        if (!box_far(s_tab.C[b], s_tab.R[b], b, om, 0) || !box_far(s_tab.C[b], s_tab.R[b], b, om, 1)) {
          lo = lo < i ? lo : i;
          hi = i + 1;
        }
      }
      if (hi <= lo) lo = hi = 0;
    }
    s_rng[b][0] = (short)lo;
    s_rng[b][1] = (short)hi;
  }
  __syncthreads();
  const bool boxes = s_tab.on != 0;
  int nfp64 = 0, npieces = 0, nboxed = 0;
  int qh = 0, qt = 0;  // ring queue head and tail (warp-uniform)
  // one queued final tetrahedron (sorted offsets ee from D0 = D0h + D0l, values ff, weight vr,
  // own far-field moments am[0..K)) on the frequencies its box (b >= 0) leaves to it, or on
  // all of them (b < 0); lanes own frequencies
  // one term of Re / Im at frequency iw
  auto add_re = [&](int iw, T v) {
    if constexpr (FX) {
      const long long t = __float2ll_rn(v * kFxScale);
      if (t) atomicAdd(&s_fx[0][iw], (unsigned long long)t);
    } else {
      kadd_t(sR[wib][iw], cR[wib][iw], v);
    }
  };
  auto add_im = [&](int iw, T v) {
    if constexpr (FX) {
      const long long t = __float2ll_rn(v * kFxScale);
      if (t) atomicAdd(&s_fx[1][iw], (unsigned long long)t);
    } else {
      kadd_t(sI[wib][iw], cI[wib][iw], v);
    }
  };
  // one round of per-lane results (iw < 0: nothing).  Fixed point: atomic adds (exact, any
  // order).  FP64: lanes that share a frequency add one at a time in lane order (the lists are
  // built in a fixed order, so the sums are reproducible), the others at once.
  auto round_add = [&](int iw, T re, T im) {
    if constexpr (FX) {
      if (iw >= 0) {
        if (re != T(0)) add_re(iw, re);
        if (im != T(0)) add_im(iw, im);
      }
    } else {
      const unsigned grp = __match_any_sync(kFull, iw >= 0 ? iw : -1 - lane);
      const int rank = __popc(grp & lt);
      const int nr = __reduce_max_sync(kFull, iw >= 0 ? rank : 0);
#pragma unroll 1
      for (int r = 0; r <= nr; ++r) {
        if (iw >= 0 && rank == r) {
          add_re(iw, re);
          if (im != T(0)) add_im(iw, im);
        }
        __syncwarp();
      }
    }
  };
  int nfb = 0;  // entries in the warp's fallback buffer
  // the fallback buffer: per-vertex table, one entry per lane and round (full rounds: the
  // buffer collects the entries of many pieces).  Lanes that share a frequency add one at a
  // time in lane order (the buffer's order is fixed, so the sums are reproducible), the others
  // at once.
  auto fallback_flush = [&]() {
    __syncwarp();
#pragma unroll 1
    for (int base = 0; base < nfb; base += 32) {
      const int k = base + lane;
      T re = T(0), im = T(0);
      int iw = -1 - lane;  // inactive lanes: keys of their own
      if (k < nfb) {
        const FbEnt<T> &o = gfb[k];
        T x[4], ff[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          x[i] = o.x[i];
          ff[i] = o.f[i];
        }
        const T vr = o.v;
        const int code = o.code;
        iw = code >> 2;
        re = vr * near_term<FP64>(x, ff, tau, nfp64);
        if ((code & 2) == 0 && x[0] < T(0) && x[3] > T(0)) {
          im = vr * delta_sum_ol(x, ff) * T(3.141592653589793);
          if (code & 1) im = -im;
        }
      }
      round_add(iw, re, im);
    }
    nfb = 0;
  };
  int nnear = 0;  // entries in the drain's near list
  // the drain's near list: the shared divided-difference table, one entry per lane and round
  // (the entries of all queued pieces packed together); lanes that share a frequency add one
  // at a time in lane order (the list's order is fixed, so the sums are reproducible).  Entries
  // the table leaves (three clustered knots, three zero knots) go, knots and all, to the
  // fallback buffer (the caller keeps room for the whole list).
  auto near_drain = [&]() {
#pragma unroll 1
    for (int base = 0; base < nnear; base += 32) {
      const int k = base + lane;
      T re = T(0), im = T(0), x[4], ff[4], vr = T(0);
      int iw = -1 - lane, ent = 0;  // inactive lanes: keys of their own
      bool left = false, neg = false;
      if (k < nnear) {
        const int code = s_near[wib][k], sl = code >> 9;
        ent = code & 511;
        T ee[4], d[4];
        const T D0h = s_qv[wib][sl][1], D0l = s_qv[wib][sl][2];
        vr = s_qv[wib][sl][0];
        if constexpr (FP64) {
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            ee[i] = s_qe[wib][sl][i];
            ff[i] = s_qf[wib][sl][i];
          }
        } else {  // one 16-byte load each
          const float4 e4 = *reinterpret_cast<const float4 *>(&s_qe[wib][sl][0]);
          const float4 f4 = *reinterpret_cast<const float4 *>(&s_qf[wib][sl][0]);
          ee[0] = e4.x, ee[1] = e4.y, ee[2] = e4.z, ee[3] = e4.w;
          ff[0] = f4.x, ff[1] = f4.y, ff[2] = f4.z, ff[3] = f4.w;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) d[i] = D0h + ee[i];
        near_knots<FP64>(ent, d, ee, D0h, D0l, s_w, s_wl, x, neg);
        // (a near entry has the frequency within two half-widths of the piece's midpoint,
        // where the moment series about the knot midpoint does not apply)
        T v;
        if constexpr (IMO) {  // the delta term alone
          if (x[0] < T(0) && x[3] > T(0)) {
            iw = ent >> 1;
            const T rs[6] = {rcp(ee[1] - ee[0]), rcp(ee[2] - ee[1]), rcp(ee[3] - ee[2]),
                             rcp(ee[2] - ee[0]), rcp(ee[3] - ee[1]), rcp(ee[3] - ee[0])};
            im = vr * delta_sum_pre(x, ff, rs) * T(3.141592653589793);
          }
        } else if (inv_sum_shared(x, ff, v)) {
          iw = ent >> 1;
          re = vr * v;
          if ((ent & 1) == 0 && x[0] < T(0) && x[3] > T(0)) {
            // reciprocal knot spans 01, 12, 23, 02, 13, 03 for the de Boor recursion (from the
            // unshifted offsets: nonnegative terms, no cancellation)
            const T rs[6] = {rcp(ee[1] - ee[0]), rcp(ee[2] - ee[1]), rcp(ee[3] - ee[2]),
                             rcp(ee[2] - ee[0]), rcp(ee[3] - ee[1]), rcp(ee[3] - ee[0])};
            im = vr * delta_sum_pre(x, ff, rs) * T(3.141592653589793);
            if (neg) im = -im;
          }
        } else {
          left = true;
        }
      }
      round_add(iw, re, im);
      const unsigned bal = __ballot_sync(kFull, left);
      if (bal) {  // warp-uniform
        if (left) {
          FbEnt<T> &o = gfb[nfb + __popc(bal & lt)];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            o.x[i] = x[i];
            o.f[i] = ff[i];
          }
          o.v = vr;
          o.code = ((ent >> 1) << 2) | ((ent & 1) << 1) | (neg ? 1 : 0);
        }
        nfb += __popc(bal);
        __syncwarp();
      }
    }
    nnear = 0;
  };
  auto eval_piece = [&](const T ee[4], const T ff[4], T vr, T D0h, T D0l, const T *am, int K, int b, int slot) {
    if constexpr (IMO) {
      // the grid frequencies inside the knot range (ascending grid: one index range, widened
      // by one on each side; the delta term's own test decides each entry)
      const T lo_d = D0h + ee[0], hi_d = D0h + ee[3];
      int a = 0, z = nw;  // first index with w > lo_d
#pragma unroll 1
      while (a < z) {
        const int mid = (a + z) >> 1;
        if (s_w[mid] > lo_d) z = mid;
        else a = mid + 1;
      }
      int c = a, e = nw;  // first index with w >= hi_d
#pragma unroll 1
      while (c < e) {
        const int mid = (c + e) >> 1;
        if (s_w[mid] >= hi_d) e = mid;
        else c = mid + 1;
      }
      const int lo = a > 0 ? a - 1 : 0, hi = c < nw ? c + 1 : nw;
#pragma unroll 1
      for (int iw = lo + lane; iw < hi; iw += 32) s_near[wib][nnear + iw - lo] = (unsigned short)((slot << 9) | (iw * 2));
      nnear += hi - lo;
      __syncwarp();
    } else {
      T d[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) d[i] = D0h + ee[i];
      const T c = D0h + (ee[0] + ee[3]) * T(0.5), half = (ee[3] - ee[0]) * T(0.5);
      const T Cb = b >= 0 ? s_tab.C[b] : T(0), Rb = b >= 0 ? s_tab.R[b] : T(0);
      const int lo = b >= 0 ? s_rng[b][0] : 0, hi = b >= 0 ? s_rng[b][1] : nw;
      // far field for both terms (Horner on the moments); near-field frequencies are
      // recorded per lane (bit it of nearm / nearp) and evaluated below in full warps
      unsigned nearm = 0u, nearp = 0u;
#pragma unroll 1
      for (int iw = lo + lane, itn = 0; iw < hi; iw += 32, ++itn) {
        const T om = s_w[iw] < T(0) ? -s_w[iw] : s_w[iw];
        T re = T(0);
        // (the + term is near only for boxes that reach below u = 0 + F R: most boxes skip it)
        const int t_hi = (b >= 0 && !(Cb < Rb * T(DynShape<FP64>::NF))) ? 0 : 1;
#pragma unroll 1
        for (int t = t_hi; t >= 0; --t) {  // the + term (t = 1), then the - term
          int kk = 0;  // own-series terms this lane needs for this term (0: none)
          if (b < 0 || !box_far(Cb, Rb, b, om, t)) {
            const T den = t ? c + om : c - om;
            const T r = quot(half, den < T(0) ? -den : den);
            if (r <= T(Num<T>::kappa_far)) kk = own_terms<T>(K, r);
            else if (t) nearp |= 1u << itn;
            else nearm |= 1u << itn;
          }
          // one trip count for the lanes of the warp (extra terms only add what lies below the
          // truncation tolerance): a convergent loop
          const int km = __reduce_max_sync(__activemask(), kk);
          if (kk > 0) re += far_eval_k(am, km, c, t ? -om : om);
        }
        if (re != T(0)) add_re(iw, vr * re);
      }
      // near field: the (frequency, term) pairs go to the drain's near list (the caller keeps
      // room for them)
      const int nit = (hi - lo + 31) >> 5;
#pragma unroll 1
      for (int itn = 0; itn < nit; ++itn) {
#pragma unroll
        for (int sgn = 0; sgn < 2; ++sgn) {
          const bool mine = ((sgn ? nearp : nearm) >> itn) & 1u;
          const unsigned bal = __ballot_sync(kFull, mine);
          if (mine) s_near[wib][nnear + __popc(bal & lt)] = (unsigned short)((slot << 9) | ((lo + itn * 32 + lane) * 2 + sgn));
          nnear += __popc(bal);
        }
      }
      __syncwarp();
    }
  };
  // evaluates n <= DC queued pieces: own far-field moments one piece per lane, then each piece
  // on its frequencies with the whole warp
  auto drain = [&](int n) {
    if (!IMO && lane < n) {
      const int sl = (qh + lane) % QC;
      T d[4], ff[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        d[i] = s_qv[wib][sl][1] + s_qe[wib][sl][i];
        ff[i] = s_qf[wib][sl][i];
      }
      s_pk[wib][lane] = far_moments<T, KM>(d, ff, scr + lane * SKM);
    }
    __syncwarp();
    // pieces one by one (p < n), the near list whenever it might not hold another piece's
    // entries and after the last piece (p == n; one call site), with room for its leftovers
#pragma unroll 1
    for (int p = 0; p <= n; ++p) {
      if (p == n ? nnear > 0 : nnear > kNearCap - 2 * kNWPass) {  // warp-uniform
        if (nfb > kFbCap - kNearCap) fallback_flush();
        near_drain();
      }
      if (p == n) break;
      const int sl = (qh + p) % QC;
      T ee[4], ff[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        ee[i] = s_qe[wib][sl][i];
        ff[i] = s_qf[wib][sl][i];
      }
      eval_piece(ee, ff, s_qv[wib][sl][0], s_qv[wib][sl][1], s_qv[wib][sl][2], scr + p * SKM, s_pk[wib][p],
                 s_qb[wib][sl], sl);
    }
    qh += n;
    __syncwarp();
  };
  int dthr = DC;  // queued pieces that trigger a drain (1: drain them all; warp-uniform)
  // one carving step: at most one final tetrahedron per lane (has).  Its box and moments, the
  // box sums (one moment index per lane, pieces in lane order), and the queue for pieces that
  // evaluate frequencies themselves.
  auto piece = [&](bool has, T ee[4], T ff[4], T vr, T D0h, T D0l) {
    int b = -1;
    if (has) {
      sort4(ee, ff);
      ++npieces;
      has = D0h + ee[3] > T(0);
    }
    if (has) {
      const T c = D0h + (ee[0] + ee[3]) * T(0.5), half = (ee[3] - ee[0]) * T(0.5);
      b = boxes ? box_of(c, half, s_tab) : -1;
      if (b >= 0) {
        const T ri = rcp(s_tab.R[b]), base = (D0h - s_tab.C[b]) + D0l;
        T e[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) e[i] = (base + ee[i]) * ri;
        if constexpr (FX) box_moments_fx(e, ff, vr, bfx + slot_base<FP64>(b), b < kBoxFine ? KF : KG);
        else box_moments_ol(e, ff, vr, scr + lane * SKF, b < kBoxFine ? KF : KG);
        ++nboxed;
      }
    }
    if constexpr (!FX) {  // FP64 box sums: one moment index per lane, pieces in lane order
      __syncwarp();
      unsigned mask = __ballot_sync(kFull, has && b >= 0);
#pragma unroll 1
      while (mask) {  // warp-uniform
        const int p = __ffs(mask) - 1;
        mask &= mask - 1u;
        const int bp = __shfl_sync(kFull, b, p);
        const int K = bp < kBoxFine ? KF : KG, base = slot_base<FP64>(bp);
#pragma unroll 1
        for (int k = lane; k < K; k += 32) acc[base + k] += scr[p * SKF + k];
      }
    }
    // (Im only: pieces whose knot range meets the pass's frequencies)
    const bool queue = has && b < kBoxFine &&
                       (!IMO || (D0h + ee[3] > s_w[0] && D0h + ee[0] < s_w[nw - 1]));
    const unsigned qm = __ballot_sync(kFull, queue);
    if (queue) {
      const int sl = (qt + __popc(qm & lt)) % QC;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        s_qe[wib][sl][i] = ee[i];
        s_qf[wib][sl][i] = ff[i];
      }
      s_qv[wib][sl][0] = vr;
      s_qv[wib][sl][1] = D0h;
      s_qv[wib][sl][2] = D0l;
      s_qb[wib][sl] = b;
    }
    qt += __popc(qm);
    __syncwarp();
    while (qt - qh >= dthr) drain(qt - qh < DC ? qt - qh : DC);
  };
  // item data of (tetrahedron l of the batch, bands m, n): a = e^m_k - eF, D = D0 + e (e_0 = 0)
  // and |M|^2 at the corners.  Mixed path: energies as FP32 hi + lo pairs, so that D0 (hi + lo)
  // and the corner offsets e come out to full FP32 relative precision whatever the size of a, b
  auto load_item = [&](int l, int m, int n, T a[4], T e[4], T f[4], T &D0h, T &D0l) {
    D0h = T(0);
    D0l = T(0);
    if constexpr (FP64) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int ck = s_c[wib][l][i], cq = s_cq[wib][l][i];
        a[i] = ((const double *)Ek)[(long long)ck * g.nb + m] - g.ef;
        e[i] = (((const double *)Ekq)[(long long)cq * g.nb + n] - g.ef) - a[i];
      }
    } else {
      float al[4], bh[4], bl[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const long long ik = (long long)s_c[wib][l][i] * g.nb + m, iq = (long long)s_cq[wib][l][i] * g.nb + n;
        a[i] = ((const float *)Ek)[ik];
        al[i] = Eklo[ik];
        bh[i] = ((const float *)Ekq)[iq];
        bl[i] = Ekqlo[iq];
      }
      float sv, tv;
      two_diff(bh[0], a[0], sv, tv);
      const float corr = tv + (bl[0] - al[0]);
      D0h = sv + corr;
      D0l = corr - (D0h - sv);
      e[0] = 0.0f;
#pragma unroll
      for (int i = 1; i < 4; ++i) {
        float sa, ta, sb, tb;
        two_diff(a[i], a[0], sa, ta);
        two_diff(bh[i], bh[0], sb, tb);
        e[i] = (sb - sa) + ((tb - ta) + ((bl[i] - bl[0]) - (al[i] - al[0])));
      }
    }
    const T *W2t = (const T *)W2;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      f[i] = cma ? T(1) : W2t[((long long)s_c[wib][l][i] * w + (m - q.lo)) * w + (n - q.lo)];
  };
  // up to 32 items, one per lane: both carvings of Sec. II as warp-uniform loops over the
  // pieces of the first and second cut, one final tetrahedron per lane and step
  // (force: at least one step, so that piece() runs and drains the queue)
  auto carve_items = [&](bool has, int l, int m, int n, bool force) {
    T a[4] = {T(0), T(0), T(0), T(0)}, e[4] = {T(0), T(0), T(0), T(0)}, f[4] = {T(0), T(0), T(0), T(0)};
    T D0h = T(0), D0l = T(0);
    if (has) load_item(l, m, n, a, e, f, D0h, D0l);
    const T vol = has ? s_vol[wib][l] : T(0);
    bool whole = false;
    if (has) {
      const T amax = fmax(fmax(a[0], a[1]), fmax(a[2], a[3]));
      const T bmin = fmin(fmin(a[0] + D0h + e[0], a[1] + D0h + e[1]), fmin(a[2] + D0h + e[2], a[3] + D0h + e[3]));
      whole = amax < T(0) && bmin > T(0);  // occupied at k and empty at k+q everywhere: no cut
    }
    // whole items emit their one piece at the first step
    Vt<T> V[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) V[i] = Vt<T>{a[i], e[i], f[i]};
    const bool cut = has && !whole;
    Vt<T> P0[4];
    T r0 = T(0);
    const int n1 = cut ? cut_piece<0>(V, 0, P0, r0) : 0;
    const int n1max = max(__reduce_max_sync(kFull, whole ? 1 : n1), force ? 1 : 0);
#pragma unroll 1
    for (int i1 = 0; i1 < n1max; ++i1) {
      Vt<T> P[4];
      T r1 = T(0);
      bool ok1 = false;
      if (cut && i1 < n1) {
        cut_piece<0>(V, i1, P, r1);
        ok1 = r1 > T(0);
#pragma unroll
        for (int i = 0; i < 4; ++i) P[i].a += D0h;  // second-cut key -(a + e) is now -b
      }
      int n2 = 0;
      if (ok1) {
        Vt<T> Qd[4];
        T rd;
        n2 = cut_piece<1>(P, 0, Qd, rd);
      }
      const int n2max = max(__reduce_max_sync(kFull, (whole && i1 == 0) ? 1 : n2), (force && i1 == 0) ? 1 : 0);
#pragma unroll 1
      for (int i2 = 0; i2 < n2max; ++i2) {
        T ee[4], ff[4], vr = T(0);
        bool okp = false;
        if (whole) {
          okp = i1 == 0 && i2 == 0;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            ee[i] = e[i];
            ff[i] = f[i];
          }
          vr = vol;
        } else if (ok1 && i2 < n2) {
          Vt<T> Qv[4];
          T r2 = T(0);
          cut_piece<1>(P, i2, Qv, r2);
          const T r = r1 * r2;
          okp = r > T(0);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            ee[i] = Qv[i].D > -D0h ? Qv[i].D : -D0h;  // clamped to D >= 0
            ff[i] = Qv[i].f;
          }
          vr = vol * r;
        } else {
#pragma unroll
          for (int i = 0; i < 4; ++i) ee[i] = ff[i] = T(0);
        }
        piece(okp, ee, ff, vr, D0h, D0l);
      }
    }
  };
  bool first = true;  // this warp's first batch writes its box partials, later ones add to them
  // batches: FP64 kernel in a fixed order per warp (batch = warp + k x warps: its FP64 sums are
  // reproducible); FP32 kernel from a launch-wide counter (its sums are exact integers, whatever
  // the order), which balances the warps' loads
  auto next_batch = [&](long long cur) -> long long {
    if constexpr (FX) {
      unsigned long long b = 0ull;
      if (lane == 0) b = atomicAdd(db.ctr, 1ull);
      return (long long)__shfl_sync(kFull, b, 0);
    } else {
      return cur < 0 ? gwarp : cur + nwarps;
    }
  };
#pragma unroll 1
  for (long long batch = next_batch(-1); batch < nbatch; batch = next_batch(batch)) {
    if constexpr (!FX) {
#pragma unroll 1
      for (int iw = lane; iw < nw; iw += 32) {
        sR[wib][iw] = T(0);
        sI[wib][iw] = T(0);
        cR[wib][iw] = T(0);
        cI[wib][iw] = T(0);
      }
    }
    const long long t = batch * 32 + lane;
    int cnt = 0;
    if (t < g.ntet) {
      long long c[4], cq[4];
      double vol;
      tet_corners(g, tet, q, t, c, cq, vol);
      int mhi = 0, nlo = g.nb;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        s_c[wib][lane][i] = (int)c[i];
        s_cq[wib][lane][i] = (int)cq[i];
        mhi = max(mhi, (int)occ[c[i]]);
        nlo = min(nlo, (int)empq[cq[i]]);
      }
      mhi = min(mhi, q.hi);
      nlo = max(nlo, q.lo);
      const int nm = mhi - q.lo, nn = q.hi - nlo;
      cnt = (nm > 0 && nn > 0) ? nm * nn : 0;
      s_vol[wib][lane] = (T)vol;
      s_nlo[wib][lane] = nlo;
      s_nn[wib][lane] = nn;
    }
    int pre = cnt;  // inclusive prefix sum over the lanes
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(kFull, pre, o);
      if (lane >= o) pre += v;
    }
    s_pre[wib][lane + 1] = pre;
    if (lane == 0) s_pre[wib][0] = 0;
    const int total = __shfl_sync(kFull, pre, 31);
    if (lane < 2) s_nl[wib][lane] = 0;
    __syncwarp();
    // Items are sorted into two per-warp lists, whole-tetrahedron items and items whose
    // tetrahedron a Fermi surface cuts, and each list is carved 32 items at a time, so that the
    // lanes of a warp mostly run the same path.
    auto drain_items = [&](bool final) {
      for (;;) {  // warp-uniform
        const int nf = s_nl[wib][0], nc = s_nl[wib][1];
        int which;
        if (nf >= 32) which = 0;
        else if (nc >= 32) which = 1;
        else if (final && nf > 0) which = 0;
        else if (final && nc > 0) which = 1;
        else if (final && qt > qh) which = 2;  // the batch's last queued pieces
        else break;
        int take = 0, code = 0;
        if (which < 2) {
          const int cntl = which ? nc : nf;
          take = cntl < 32 ? cntl : 32;
          if (lane < take) code = s_list[wib][which][cntl - take + lane];
          __syncwarp();
          if (lane == 0) s_nl[wib][which] = cntl - take;
          __syncwarp();
        }
        dthr = which == 2 ? 1 : DC;
        const unsigned u = (unsigned)code;
        carve_items(lane < take, (int)(u >> 24), (int)((u >> 12) & 0xFFFu), (int)(u & 0xFFFu), which == 2);
      }
      dthr = DC;
    };
    for (int base = 0;; base += 32) {  // warp-uniform; the pass after the last items drains
      const bool last = base >= total;
      const int it = base + lane;
      int kind = -1, code = 0;  // 0: whole tetrahedron (likely), 1: cut, -1: nothing to do
      if (it < total) {
        int lo_ = 0, hi_ = 32;  // owner: largest l with s_pre[l] <= it
#pragma unroll
        for (int step = 0; step < 5; ++step) {
          const int mid = (lo_ + hi_) >> 1;
          if (s_pre[wib][mid] <= it) lo_ = mid;
          else hi_ = mid;
        }
        const int l = lo_;
        const int loc = it - s_pre[wib][l];
        const int nn = s_nn[wib][l];
        const int mo = div_small(loc, nn, q.hi - q.lo);
        const int m = q.lo + mo, n = s_nlo[wib][l] + (loc - mo * nn);
        if (!(q.gamma && m == n)) {  // intraband at Gamma: replaced by the DOS limit
          T amin = T(1e30), amax = T(-1e30), bmin = T(1e30), bmax = T(-1e30);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            T a, b;
            if constexpr (FP64) {
              a = ((const double *)Ek)[(long long)s_c[wib][l][i] * g.nb + m] - g.ef;
              b = ((const double *)Ekq)[(long long)s_cq[wib][l][i] * g.nb + n] - g.ef;
            } else {
              a = ((const float *)Ek)[(long long)s_c[wib][l][i] * g.nb + m];
              b = ((const float *)Ekq)[(long long)s_cq[wib][l][i] * g.nb + n];
            }
            amin = a < amin ? a : amin;
            amax = a > amax ? a : amax;
            bmin = b < bmin ? b : bmin;
            bmax = b > bmax ? b : bmax;
          }
          if (amin < T(0) && bmax > T(0)) {
            kind = (amax < T(0) && bmin > T(0)) ? 0 : 1;
            code = (l << 24) | (m << 12) | n;
          }
        }
      }
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const unsigned bal = __ballot_sync(kFull, kind == k);
        if (kind == k) s_list[wib][k][s_nl[wib][k] + __popc(bal & lt)] = code;
        __syncwarp();
        if (lane == 0) s_nl[wib][k] += __popc(bal);
        __syncwarp();
      }
      drain_items(last);
      if (last) break;
    }
    qh = qt = 0;  // (the last pass of drain_items emptied the queue)
    if constexpr (!FX) {
      if (nfb > 0) fallback_flush();  // warp-uniform
      __syncwarp();
#pragma unroll 1
      for (int iw = lane; iw < nw; iw += 32) {
        db.partR[batch * nw + iw] = (double)sR[wib][iw] + (double)cR[wib][iw];
        db.partI[batch * nw + iw] = (double)sI[wib][iw] + (double)cI[wib][iw];
      }
      // this batch's box sums into the warp's FP64 partials (a fixed order: bitwise reproducible)
      if (boxes) {
#pragma unroll 1
        for (int i = lane; i < NS; i += 32) {
          const double v = (double)acc[i];
          gpart[i] = first ? v : gpart[i] + v;
          acc[i] = T(0);
        }
      }
    }
    first = false;
    __syncwarp();
  }
  if constexpr (FX) {
    // the warp's remaining fallback entries, then the CTA's fixed-point sums into its rows
    if (nfb > 0) fallback_flush();  // warp-uniform
    __syncthreads();
    unsigned long long *row = db.fx + (size_t)blockIdx.x * 2 * kNWPass;
    unsigned long long *brow = (unsigned long long *)db.box_part + (size_t)blockIdx.x * NS;
#pragma unroll 1
    for (int i = threadIdx.x; i < 2 * kNWPass; i += blockDim.x) row[i] = s_fx[i / kNWPass][i % kNWPass];
    if constexpr (!IMO) {
#pragma unroll 1
      for (int i = threadIdx.x; i < NS; i += blockDim.x) brow[i] = bfx[i];
    }
  } else {
    if (boxes && first)  // a warp without batches
#pragma unroll 1
      for (int i = lane; i < NS; i += 32) gpart[i] = 0.0;
  }
  if (counters) {
    unsigned long long a = (unsigned long long)npieces, b = (unsigned long long)nfp64,
                       x = (unsigned long long)nboxed;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(kFull, a, o);
      b += __shfl_xor_sync(kFull, b, o);
      x += __shfl_xor_sync(kFull, x, o);
    }
    if (lane == 0) {
      atomicAdd(&counters[0], a);  // each lane counted its own pieces
      atomicAdd(&counters[1], b);
      atomicAdd(&counters[3], x);
    }
  }
}

// box totals: slot i summed over the rows of the weight launch (FP64 kernel: per-warp FP64
// partials, in warp order; FP32 kernel: per-CTA fixed-point rows, summed exactly)
template <bool FP64>
__global__ void __launch_bounds__(256) k_box_sum(const double *__restrict__ part, int nrows, double *__restrict__ tot) {
  constexpr int NS = box_slots<FP64>();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NS) return;
  if constexpr (FP64) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int wv = 0;
    for (; wv + 3 < nrows; wv += 4) {
      s0 += part[(size_t)wv * NS + i];
      s1 += part[(size_t)(wv + 1) * NS + i];
      s2 += part[(size_t)(wv + 2) * NS + i];
      s3 += part[(size_t)(wv + 3) * NS + i];
    }
    for (; wv < nrows; ++wv) s0 += part[(size_t)wv * NS + i];
    tot[i] = (s0 + s1) + (s2 + s3);
  } else {
    const unsigned long long *fx = (const unsigned long long *)part;
    unsigned long long a = 0ull;
    for (int r = 0; r < nrows; ++r) a += fx[(size_t)r * NS + i];
    tot[i] = (double)(long long)a * kFxUnit;
  }
}

// FP32 kernel: Re and Im per frequency from the CTAs' fixed-point rows (exact sums) into row 0
// of the partials
__global__ void __launch_bounds__(256) k_fx_rows(const unsigned long long *__restrict__ fx, int nrows, int nw,
                                                 double *__restrict__ partR, double *__restrict__ partI) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * nw) return;
  const int term = i / nw, iw = i % nw;
  unsigned long long a = 0ull;
  for (int r = 0; r < nrows; ++r) a += fx[((size_t)r * 2 + term) * kNWPass + iw];
  (term ? partI : partR)[iw] = (double)(long long)a * kFxUnit;
}

// far[iw]: the boxes' share of Re at frequency iw (FP64 evaluation of the multipoles); one
// block per frequency, fixed-order reduction
template <bool FP64>
__global__ void __launch_bounds__(128) k_box_eval(const double *__restrict__ omega, const void *__restrict__ tabp,
                                                  const double *__restrict__ tot, double *__restrict__ far) {
  using T = typename std::conditional<FP64, double, float>::type;
  using S = DynShape<FP64>;
  const BoxTab<T> &tb = *(const BoxTab<T> *)tabp;
  const int iw = blockIdx.x;
  const double u = fabs(omega[iw]);
  const T wT = (T)omega[iw];
  const T om = wT < T(0) ? -wT : wT;
  double v = 0.0;
  if (tb.on) {
    for (int b = threadIdx.x; b < kBoxes; b += blockDim.x) {
      const int K = b < kBoxFine ? S::KF : S::KG;
      const double *M = tot + slot_base<FP64>(b);
      const double C = (double)tb.C[b], R = (double)tb.R[b];
      for (int term = 0; term < 2; ++term) {
        if (!box_far(tb.C[b], tb.R[b], b, om, term)) continue;
        const double den = term ? C + u : C - u;
        const double mz = -R / den;
        double s = M[K - 1];
        for (int k = K - 2; k >= 0; --k) s = s * mz + M[k];
        v += s / den;
      }
    }
  }
  __shared__ double red[4];
  v = grid::warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) far[iw] = (red[0] + red[1]) + (red[2] + red[3]);
}

template <bool FP64> size_t dyn_smem() {
  return FP64 ? (size_t)DynShape<FP64>::warps * box_slots<FP64>() * sizeof(double)
              : (size_t)box_slots<FP64>() * sizeof(unsigned long long);
}

}  // namespace

int dynamic_max_nw() { return kNWPass; }
int dynamic_warps_per_cta(int fp64) { return fp64 ? DynShape<true>::warps : DynShape<false>::warps; }
size_t dynamic_box_slots(int fp64) { return fp64 ? box_slots<true>() : box_slots<false>(); }
size_t dynamic_fx_bytes(int nblocks) { return (size_t)nblocks * 2 * kNWPass * sizeof(unsigned long long); }
size_t dynamic_fb_bytes(int fp64) {
  return (size_t)kFbCap * (fp64 ? sizeof(FbEnt<double>) : sizeof(FbEnt<float>));
}
size_t dynamic_box_tab_bytes() {
  return sizeof(BoxTab<double>) > sizeof(BoxTab<float>) ? sizeof(BoxTab<double>) : sizeof(BoxTab<float>);
}

cudaError_t dynamic_prepare() {
  cudaError_t e = cudaFuncSetAttribute(k_dynamic<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)dyn_smem<true>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_dynamic<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)dyn_smem<false>());
}

cudaError_t launch_dynamic(const Grid &g, const Tet &tet, const void *Ek, const void *Ekq, const Q &q,
                           const void *W2, int cma, int fp64, float tau, const short *occ, const short *empq,
                           const double *omega, int nw, const DynBufs &db, int nblocks,
                           unsigned long long *counters, cudaStream_t s, const float *Eklo,
                           const float *Ekqlo, int *rows) {
  if (nw > kNWPass || nw <= 0 || nblocks <= 0) return cudaErrorInvalidValue;
  if (!fp64 && (!Eklo || !Ekqlo)) return cudaErrorInvalidValue;
  if (!db.box_tab || !db.box_part || !db.box_tot || !db.far || !db.fb || !db.fx || !db.ctr)
    return cudaErrorInvalidValue;
  if (fp64) {
    const int nwarps = nblocks * DynShape<true>::warps;
    k_box_setup<double><<<1, 256, 0, s>>>(omega, nw, (BoxTab<double> *)db.box_tab);
    k_dynamic<true><<<nblocks, DynShape<true>::threads, dyn_smem<true>(), s>>>(
        g, tet, Ek, Ekq, q, W2, cma, tau, occ, empq, omega, nw, db, Eklo, Ekqlo, counters);
    k_box_sum<true><<<(box_slots<true>() + 255) / 256, 256, 0, s>>>(db.box_part, nwarps, db.box_tot);
    k_box_eval<true><<<nw, 128, 0, s>>>(omega, db.box_tab, db.box_tot, db.far);
    *rows = (int)((g.ntet + 31) / 32);
  } else {
    cudaError_t e = cudaMemsetAsync(db.ctr, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    k_box_setup<float><<<1, 256, 0, s>>>(omega, nw, (BoxTab<float> *)db.box_tab);
    k_dynamic<false><<<nblocks, DynShape<false>::threads, dyn_smem<false>(), s>>>(
        g, tet, Ek, Ekq, q, W2, cma, tau, occ, empq, omega, nw, db, Eklo, Ekqlo, counters);
    k_box_sum<false><<<(box_slots<false>() + 255) / 256, 256, 0, s>>>(db.box_part, nblocks, db.box_tot);
    k_box_eval<false><<<nw, 128, 0, s>>>(omega, db.box_tab, db.box_tot, db.far);
    k_fx_rows<<<(2 * nw + 255) / 256, 256, 0, s>>>(db.fx, nblocks, nw, db.partR, db.partI);
    *rows = 1;
  }
  return cudaGetLastError();
}

// Im only (the Kramers-Kronig route): the delta term on an ascending grid of w >= 0
cudaError_t launch_dynamic_im(const Grid &g, const Tet &tet, const void *Ek, const void *Ekq, const Q &q,
                              const void *W2, int cma, int fp64, float tau, const short *occ, const short *empq,
                              const double *omega, int nw, const DynBufs &db, int nblocks,
                              unsigned long long *counters, cudaStream_t s, const float *Eklo,
                              const float *Ekqlo, int *rows) {
  if (nw > kNWPass || nw <= 0 || nblocks <= 0) return cudaErrorInvalidValue;
  if (!fp64 && (!Eklo || !Ekqlo)) return cudaErrorInvalidValue;
  if (!db.fb || !db.fx || !db.ctr) return cudaErrorInvalidValue;
  if (fp64) {
    k_dynamic<true, true><<<nblocks, DynShape<true>::threads, 0, s>>>(g, tet, Ek, Ekq, q, W2, cma, tau, occ, empq,
                                                                       omega, nw, db, Eklo, Ekqlo, counters);
    *rows = (int)((g.ntet + 31) / 32);
  } else {
    cudaError_t e = cudaMemsetAsync(db.ctr, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    k_dynamic<false, true><<<nblocks, DynShape<false>::threads, 0, s>>>(g, tet, Ek, Ekq, q, W2, cma, tau, occ, empq,
                                                                         omega, nw, db, Eklo, Ekqlo, counters);
    k_fx_rows<<<(2 * nw + 255) / 256, 256, 0, s>>>(db.fx, nblocks, nw, db.partR, db.partI);
    *rows = 1;
  }
  return cudaGetLastError();
}

int dynamic_max_ctas_per_sm(int fp64) {
  int nb = 0;
  cudaError_t e = fp64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_dynamic<true>, DynShape<true>::threads,
                                                                      dyn_smem<true>())
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_dynamic<false>,
                                                                      DynShape<false>::threads, dyn_smem<false>());
  return (e != cudaSuccess || nb < 1) ? 1 : nb;
}

int dynamic_persistent_blocks(int fp64) { return dynamic_max_ctas_per_sm(fp64) * device_sms(); }

}  // namespace chi0int
