// chi0_kernels.cu -- sm_103a kernels of the doubly carved tetrahedron method.
//
//  k_overlap_small / k_overlap  (Eq. 1 matrix elements, tight-binding form of the Sec. III
//             footnote) on the CUDA cores: W2[c][m][n] = |sum_o conj(C_k[o][m]) C_{k+q}[o][n]|^2
//             at every k corner (the tensor-core form is in chi0_overlap_tc.cu).
//  k_bands    E - eF in FP32 (hi, and lo for the dynamic kernel) and the occupied / empty band
//             bounds of every corner.
//  k_static   persistent warps take batches of 32 tetrahedra; a batch's (m, n) rectangles
//             (occupied band m at some corner, empty band n at some corner of k+q) form one
//             item list, sorted into whole-tetrahedron and cut items and evaluated 32 at a
//             time: the two carvings of Sec. II and the closed-form 2/D integral (Eq. 1 at
//             w = 0) by its midpoint series; other pieces are queued for k_static_tab.
//             Per-batch FP64 partial sums.
//  (the dynamic weights, Eqs. 1-3, are in chi0_dynamic.cu)
//  k_dos      Gamma: the intraband q -> 0 limit, tetrahedron DOS at eF (Sec. III).
//  k_reduce   deterministic fixed-order sum of the batch partials.
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "chi0_grid.cuh"
#include "chi0_internal.h"
#include "chi0_math.cuh"

using namespace chi0dev;

namespace chi0int {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kSMs = 152;                 // default when the device cannot be queried
constexpr int kStaticBlocks = kSMs * 8;   // fixed grid of the DOS kernel (its partials)
// band-pair output: 64-bit fixed point in units of 2^-50 (|pair totals| < 2^13; one rounding
// of 2^-51 per term)
constexpr double kPairScale = 1125899906842624.0;  // 2^50
__device__ __forceinline__ void pair_add(unsigned long long *pairs, int idx, double v) {
  atomicAdd(&pairs[idx], (unsigned long long)__double2ll_rn(v * kPairScale));
}
using grid::kFull;
using grid::div_small;
using grid::tet_corners;
using grid::warp_sum;

// double -> float rounded to nearest even by integer operations (keeps the conversion of
// complex128 inputs off the FP64 pipe); magnitudes below 2^-126 flush to zero
__device__ __forceinline__ float d2f_int(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(u >> 32);
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7f800000u | (((u << 12) != 0ull && e > 1000) ? 0x400000u : 0u));
  const unsigned long long mant = u & 0xFFFFFFFFFFFFFull;
  unsigned m = (unsigned)(mant >> 29);
  const unsigned rem = (unsigned)(mant & 0x1FFFFFFFull);
  m += (rem > 0x10000000u) | ((rem == 0x10000000u) & (m & 1u));
  return __uint_as_float(sign | (((unsigned)e << 23) + m));  // a mantissa carry rounds into the exponent
}

template <typename T> __device__ __forceinline__ T cvt(double x);
template <> __device__ __forceinline__ float cvt<float>(double x) { return d2f_int(x); }
template <typename T> __device__ __forceinline__ T cvt(float x) { return (T)x; }

__device__ __forceinline__ void block_sum_store(double v, double *out) {
  __shared__ double red[kWarps];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  if (lane == 0) red[wib] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < kWarps; ++i) s += red[i];
    *out = s;
  }
}

// ---------------------------------------------------------------- overlap
// Thread per output (m, n) at a corner: general sizes.
template <typename CT, typename T>
__global__ void __launch_bounds__(kThreads) k_overlap(Grid g, const CT *__restrict__ C,
                                                       const CT *__restrict__ Cqx, Q q, T *__restrict__ W2) {
  const int w = q.hi - q.lo;
  const long long total = g.nc * (long long)w * w;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long c = idx / ((long long)w * w);
    const int r = (int)(idx - c * w * w);
    const int mm = r / w, nn = r - (r / w) * w;
    const long long ck = Cqx ? c : shift_corner(g, c, q.shift);
    const CT *Cb = Cqx ? Cqx : C;
    T re = T(0), im = T(0);
    for (int o = 0; o < g.norb; ++o) {
      const CT x = C[(c * g.norb + o) * g.nb + q.lo + mm];
      const CT y = Cb[(ck * g.norb + o) * g.nb + q.lo + nn];
      const T xr = (T)x.x, xi = (T)x.y, yr = (T)y.x, yi = (T)y.y;
      re += xr * yr + xi * yi;  // conj(x) * y
      im += xr * yi - xi * yr;
    }
    W2[idx] = re * re + im * im;
  }
}

// Warp per corner for small blocks (norb * w <= kOvlSmall): both eigenvector blocks
// C_k[:, lo:hi] and C_{k+q}[:, lo:hi] are read once, coalesced, into shared memory in
// the arithmetic precision, then the lanes form the w x w |overlap|^2 block.
constexpr int kOvlSmall = 256;
template <typename CT, typename CTq, typename T>
__global__ void __launch_bounds__(kThreads) k_overlap_small(Grid g, const CT *__restrict__ C,
                                                             const CTq *__restrict__ Cb, int explicit_q, Q q,
                                                             T *__restrict__ W2) {
  __shared__ T sA[kWarps][2][kOvlSmall], sB[kWarps][2][kOvlSmall];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int w = q.hi - q.lo, no = g.norb, nel = no * w;
  for (long long c = (long long)blockIdx.x * kWarps + wib; c < g.nc; c += (long long)gridDim.x * kWarps) {
    const long long ck = explicit_q ? c : shift_corner(g, c, q.shift);
    for (int i = lane; i < nel; i += 32) {
      const int o = i / w, mm = i - o * w;
      const CT x = C[(c * no + o) * g.nb + q.lo + mm];
      const CTq y = Cb[(ck * no + o) * g.nb + q.lo + mm];
      sA[wib][0][i] = cvt<T>(x.x);
      sA[wib][1][i] = cvt<T>(x.y);
      sB[wib][0][i] = cvt<T>(y.x);
      sB[wib][1][i] = cvt<T>(y.y);
    }
    __syncwarp();
    for (int out = lane; out < w * w; out += 32) {
      const int mm = out / w, nn = out - mm * w;
      T re = T(0), im = T(0);
      for (int o = 0; o < no; ++o) {
        const T xr = sA[wib][0][o * w + mm], xi = sA[wib][1][o * w + mm];
        const T yr = sB[wib][0][o * w + nn], yi = sB[wib][1][o * w + nn];
        re += xr * yr + xi * yi;  // conj(x) * y
        im += xr * yi - xi * yr;
      }
      W2[c * w * w + out] = re * re + im * im;
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------- band bounds per corner
// occ[c] = 1 + highest band with e < eF at corner c (0 if none): bands m >= occ[c] are empty
// there.  emp[c] = lowest band with e > eF (nb if none): bands n < emp[c] are not empty.
// E32 (optional) receives the energies relative to eF in FP32 for the mixed-precision path.
__global__ void __launch_bounds__(kThreads) k_bands(const double *__restrict__ E, long long nc, int nb,
                                                    double ef, short *__restrict__ occ,
                                                    short *__restrict__ emp, float *__restrict__ E32,
                                                    float *__restrict__ E32lo) {
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < nc;
       c += (long long)gridDim.x * blockDim.x) {
    int o = 0, e = nb;
    for (int b = 0; b < nb; ++b) {
      const double x = E[c * nb + b] - ef;
      if (x < 0.0) o = b + 1;
      if (x > 0.0 && e == nb) e = b;
      if (E32) E32[c * nb + b] = (float)x;
      if (E32lo) E32lo[c * nb + b] = (float)(x - (double)(float)x);
    }
    occ[c] = (short)o;
    emp[c] = (short)e;
  }
}

// ---------------------------------------------------------------- static weights
// Three kernels per q:
//  k_static      persistent warps take batches of 32 tetrahedra from an atomic counter; a
//                batch's (m, n) rectangles are flattened into one item list shared by the
//                lanes; carving; final tetrahedra whose knots fit the short series are
//                evaluated on the spot (compact hot loop), the others are queued in the
//                batch's region of a global queue
//  k_static_tab  one warp per batch region: long series or divided-difference table
// Every batch has its own partial sums (series part, queued part), added in a fixed
// order, so the result does not depend on which warp took which batch.
constexpr int kTabCap = 64;  // queued final tetrahedra per batch (plans; StaticBufs::tcap at run time)

template <typename T> struct Piece {
  T d[4], f[4], w;
  int code;  // bit 0: evaluate in FP64 (near-degenerate knots); bits 1..: band pair (m - lo) w + (n - lo)
};

// compensated (Neumaier) accumulator in the kernel's precision
template <typename T> struct Acc {
  T s = T(0), c = T(0);
  __device__ __forceinline__ void add(T x) {
    const T t = s + x;
    if (tabs(s) >= tabs(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// a queued piece evaluated where it is (only when its batch region is full)
template <bool FP64>
__device__ __noinline__ double piece_eval(const Piece<typename std::conditional<FP64, double, float>::type> &pc,
                                          float tau, int &nfp64) {
  if constexpr (FP64) {
    return pc.w * inv_sum_fast(pc.d, pc.f);
  } else {
    float x[4];
    if (!mixed_knots(x, pc.d, tau)) return (double)(pc.w * inv_sum_long(x, pc.f));
    ++nfp64;
    double xd[4] = {x[0], x[1], x[2], x[3]}, fd[4] = {pc.f[0], pc.f[1], pc.f[2], pc.f[3]};
    return (double)pc.w * inv_sum_table(xd, fd);
  }
}


// Block shapes of k_static (threads, resident blocks per SM the register allocation must
// allow): the autotuner picks one per plan.  FP32: 256 x 2 (128 registers), 128 x 3 (170),
// 256 x 1 (255); FP64: 256 x 1.
template <bool FP64, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    k_static(Grid g, Tet tet, const void *__restrict__ Ek, const void *__restrict__ Ekq, Q q,
             const void *__restrict__ W2, int cma, float tau, const short *__restrict__ occ,
             const short *__restrict__ empq, StaticBufs sb, unsigned long long *__restrict__ counters) {
  using T = typename std::conditional<FP64, double, float>::type;
  constexpr int kWarps = NT / 32;  // warps of this block shape
  __shared__ int s_c[kWarps][32][4], s_cq[kWarps][32][4];
  __shared__ T s_vol[kWarps][32];
  __shared__ int s_nlo[kWarps][32], s_nn[kWarps][32], s_pre[kWarps][33];
  __shared__ int s_qn[kWarps];
  __shared__ int s_list[kWarps][2][64], s_nl[kWarps][2];  // items l << 24 | m << 12 | n
  Piece<T> *tq = (Piece<T> *)sb.tq;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int w = q.hi - q.lo;
  const long long nbatch = (g.ntet + 31) / 32;
  int nfp64 = 0, npieces = 0, nover = 0;
  for (;;) {
    int batch = 0;
    if (lane == 0) batch = atomicAdd(sb.next, 1);
    batch = __shfl_sync(kFull, batch, 0);
    if (batch >= nbatch) break;
    if (lane == 0) s_qn[wib] = 0;
    Acc<T> acc;
    double acc_q = 0.0;  // pieces evaluated in place when the batch region is full
    // one tetrahedron per lane: corners, volume, band rectangle
    const long long t = (long long)batch * 32 + lane;
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
      s_vol[wib][lane] = (T)(2.0 * vol);
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
    __syncwarp();
    // final tetrahedron -> series on the spot, or the batch's queue region
    auto emit = [&](T r, T d[4], T ff[4], T vol2, int pidx) {
      sort4(d, ff);
      ++npieces;
      if (series_ok(d, T(Num<T>::kappa))) {
        const T v = vol2 * r * series_sum(d, ff);
        acc.add(v);
        if (sb.pairs) pair_add(sb.pairs, pidx, (double)v);
        return;
      }
      Piece<T> pc;
      int fp = 0;
      if constexpr (FP64) {
#pragma unroll
        for (int i = 0; i < 4; ++i) pc.d[i] = d[i];
      } else {
        fp = mixed_knots(pc.d, d, tau) ? 1 : 0;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) pc.f[i] = ff[i];
      pc.w = vol2 * r;
      pc.code = (pidx << 1) | fp;
      const int slot = atomicAdd(&s_qn[wib], 1);
      if (slot < sb.tcap) {
        nfp64 += fp;
        tq[(long long)batch * sb.tcap + slot] = pc;
      } else {
        ++nover;
        const double v = piece_eval<FP64>(pc, tau, nfp64);
        acc_q += v;
        if (sb.pairs) pair_add(sb.pairs, pidx, v);
      }
    };
    // corner data of item (tetrahedron l of the batch, bands m, n)
    auto load = [&](int l, int m, int n, T a[4], T b[4]) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int ck = s_c[wib][l][i], cq = s_cq[wib][l][i];
        if constexpr (FP64) {
          a[i] = ((const double *)Ek)[(long long)ck * g.nb + m] - g.ef;
          b[i] = ((const double *)Ekq)[(long long)cq * g.nb + n] - g.ef;
        } else {
          a[i] = ((const float *)Ek)[(long long)ck * g.nb + m];
          b[i] = ((const float *)Ekq)[(long long)cq * g.nb + n];
        }
      }
    };
    auto load_f = [&](int l, int m, int n, T f[4]) {
      const T *W2t = (const T *)W2;
#pragma unroll
      for (int i = 0; i < 4; ++i)
        f[i] = cma ? T(1) : W2t[((long long)s_c[wib][l][i] * w + (m - q.lo)) * w + (n - q.lo)];
    };
    // Items are sorted into two per-warp lists, whole-tetrahedron items (most of them: one
    // final tetrahedron, no cut) and items whose tetrahedron a Fermi surface cuts, and each
    // list is evaluated 32 items at a time, so that the lanes of a warp run the same path
    // (the few carving lanes no longer hold up the rest).  One call site of the carving.
    auto drain = [&](bool final) {
      for (;;) {  // warp-uniform
        const int nf = s_nl[wib][0], nc = s_nl[wib][1];
        int which;
        if (nf >= 32) which = 0;
        else if (nc >= 32) which = 1;
        else if (final && nf > 0) which = 0;
        else if (final && nc > 0) which = 1;
        else break;
        const int cnt = which ? nc : nf;
        const int take = cnt < 32 ? cnt : 32;
        int e = 0;
        if (lane < take) e = s_list[wib][which][cnt - take + lane];
        __syncwarp();
        if (lane == 0) s_nl[wib][which] = cnt - take;
        __syncwarp();
        if (lane < take) {
          const unsigned u = (unsigned)e;
          const int l = (int)(u >> 24), m = (int)((u >> 12) & 0xFFFu), n = (int)(u & 0xFFFu);
          T a[4], b[4], f[4];
          load(l, m, n, a, b);
          load_f(l, m, n, f);
          const T vol2 = s_vol[wib][l];
          const int pidx = (m - q.lo) * w + (n - q.lo);
          carve2<T>(a, b, f, [&](T r, T d[4], T ff[4]) { emit(r, d, ff, vol2, pidx); });
        }
      }
    };
    if (lane < 2) s_nl[wib][lane] = 0;
    __syncwarp();
    for (int base = 0;; base += 32) {  // warp-uniform; the pass after the last items drains
      const bool last = base >= total;
      const int it = base + lane;
      int kind = -1, code = 0;  // 0: whole tetrahedron, 1: cut, -1: nothing to do
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
          T a[4], b[4];
          load(l, m, n, a, b);
          T amin = a[0], amax = a[0], bmin = b[0], bmax = b[0];
#pragma unroll
          for (int i = 1; i < 4; ++i) {
            amin = a[i] < amin ? a[i] : amin;
            amax = a[i] > amax ? a[i] : amax;
            bmin = b[i] < bmin ? b[i] : bmin;
            bmax = b[i] > bmax ? b[i] : bmax;
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
        if (kind == k) s_list[wib][k][s_nl[wib][k] + __popc(bal & ((1u << lane) - 1u))] = code;
        __syncwarp();
        if (lane == 0) s_nl[wib][k] += __popc(bal);
        __syncwarp();
      }
      drain(last);
      if (last) break;
    }
    __syncwarp();
    const double v = warp_sum(acc.value() + acc_q);
    if (lane == 0) {
      sb.partial[batch] = v;
      sb.tq_n[batch] = min(s_qn[wib], sb.tcap);
    }
    __syncwarp();
  }
  if (counters) {
    unsigned long long a = (unsigned long long)npieces, b = (unsigned long long)nfp64,
                       o2 = (unsigned long long)nover;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(kFull, a, o);
      b += __shfl_xor_sync(kFull, b, o);
      o2 += __shfl_xor_sync(kFull, o2, o);
    }
    if (lane == 0) {
      atomicAdd(&counters[0], a);
      atomicAdd(&counters[1], b);
      if (o2) atomicAdd(&counters[2], o2);
    }
  }
}

// one warp per batch region: queued pieces in slot order
template <bool FP64>
__global__ void __launch_bounds__(kThreads) k_static_tab(long long nbatch, StaticBufs sb) {
  using T = typename std::conditional<FP64, double, float>::type;
  const Piece<T> *tq = (const Piece<T> *)sb.tq;
  const int lane = threadIdx.x & 31;
  for (long long b = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nbatch;
       b += ((long long)gridDim.x * blockDim.x) >> 5) {
    const int n = sb.tq_n[b];
    double acc = 0.0;
    unsigned any64 = 0u;
    for (int slot = lane; slot < n; slot += 32) {
      const Piece<T> pc = tq[b * sb.tcap + slot];
      double v = 0.0;
      if constexpr (FP64) {
        v = pc.w * inv_sum_fast(pc.d, pc.f);
      } else if (pc.code & 1) {
        any64 = 1u;  // near-degenerate knots: the FP64 table, below
        continue;
      } else {
        v = (double)(pc.w * inv_sum_long(pc.d, pc.f));
      }
      acc += v;
      if (sb.pairs) pair_add(sb.pairs, pc.code >> 1, v);
    }
    if constexpr (!FP64) {
      // FP64 entries (rare): four lanes, one vertex j each, to cut the FP64 latency
      if (__any_sync(kFull, any64)) {
        for (int slot = 0; slot < n; ++slot) {
          const Piece<T> pc = tq[b * sb.tcap + slot];
          if (!(pc.code & 1)) continue;
          double t = 0.0;
          if (lane < 4) {
            double xd[4] = {pc.d[0], pc.d[1], pc.d[2], pc.d[3]}, fd[4] = {pc.f[0], pc.f[1], pc.f[2], pc.f[3]};
            t = inv_term_table(xd, fd, lane);
          }
          t += __shfl_xor_sync(kFull, t, 1);
          t += __shfl_xor_sync(kFull, t, 2);
          if (lane == 0) {
            acc += (double)pc.w * t;
            if (sb.pairs) pair_add(sb.pairs, pc.code >> 1, (double)pc.w * t);
          }
        }
      }
    }
    const double v = warp_sum(acc);
    if (lane == 0) sb.partial[nbatch + b] = v;
  }
}

// The queued pieces compacted over all batches (one piece per thread instead of one batch per
// warp: a batch holds ~12 of its 64 slots, so the per-batch walk ran 6.6 of 32 lanes):
// exclusive scan of the per-batch counts, evaluation into vals[i], and a per-batch sum of
// vals over the batch's segment in a fixed order (results independent of the schedule).
__global__ void __launch_bounds__(1024) k_tab_scan(const int *__restrict__ n, long long nbatch,
                                                    int *__restrict__ off) {
  __shared__ long long part[1024];
  const long long per = (nbatch + 1023) / 1024;
  const long long b0 = threadIdx.x * per, b1 = b0 + per < nbatch ? b0 + per : nbatch;
  long long sum = 0;
  for (long long b = b0; b < b1; ++b) sum += n[b];
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {  // inclusive scan of the thread sums
    const long long v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  long long run = threadIdx.x ? part[threadIdx.x - 1] : 0;
  for (long long b = b0; b < b1; ++b) {
    off[b] = (int)run;
    run += n[b];
  }
  if (threadIdx.x == 1023) off[nbatch] = (int)part[1023];
}

template <bool FP64>
__global__ void __launch_bounds__(kThreads) k_tab_eval(long long nbatch, StaticBufs sb) {
  using T = typename std::conditional<FP64, double, float>::type;
  const Piece<T> *tq = (const Piece<T> *)sb.tq;
  const int total = sb.off[nbatch];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    long long lo = 0, hi = nbatch;  // batch: largest b with off[b] <= i
    while (hi - lo > 1) {
      const long long mid = (lo + hi) >> 1;
      if (sb.off[mid] <= i) lo = mid;
      else hi = mid;
    }
    const Piece<T> pc = tq[lo * sb.tcap + (i - sb.off[lo])];
    double v;
    if constexpr (FP64) {
      v = pc.w * inv_sum_fast(pc.d, pc.f);
    } else if (pc.code & 1) {  // near-degenerate knots: the FP64 table
      double xd[4] = {pc.d[0], pc.d[1], pc.d[2], pc.d[3]}, fd[4] = {pc.f[0], pc.f[1], pc.f[2], pc.f[3]};
      v = (double)pc.w * inv_sum_table(xd, fd);
    } else {
      v = (double)(pc.w * inv_sum_long(pc.d, pc.f));
    }
    sb.vals[i] = v;
    if (sb.pairs) pair_add(sb.pairs, pc.code >> 1, v);
  }
}

__global__ void __launch_bounds__(kThreads) k_tab_sum(long long nbatch, StaticBufs sb) {
  const int lane = threadIdx.x & 31;
  for (long long b = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nbatch;
       b += ((long long)gridDim.x * blockDim.x) >> 5) {
    double acc = 0.0;
    for (int i = sb.off[b] + lane; i < sb.off[b + 1]; i += 32) acc += sb.vals[i];
    const double v = warp_sum(acc);
    if (lane == 0) sb.partial[nbatch + b] = v;
  }
}

// ---------------------------------------------------------------- Gamma DOS term
__global__ void __launch_bounds__(kThreads) k_dos(Grid g, Tet tet, const double *__restrict__ E, int lo,
                                                   int hi, double *__restrict__ partial,
                                                   unsigned long long *__restrict__ pairs) {
  const int w = hi - lo;
  const long long total = g.ntet * (long long)w;
  Q q0{};
  q0.Eq = E;  // corners at k only
  double acc = 0.0;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long t = idx / w;
    const int band = lo + (int)(idx - t * w);
    long long c[4], cq[4];
    double vol;
    tet_corners(g, tet, q0, t, c, cq, vol);
    const double v = vol * dos4(E[c[0] * g.nb + band] - g.ef, E[c[1] * g.nb + band] - g.ef,
                                E[c[2] * g.nb + band] - g.ef, E[c[3] * g.nb + band] - g.ef);
    acc += v;
    if (pairs && v != 0.0) pair_add(pairs, (band - lo) * (w + 1), v);  // the intraband pair (m, m)
  }
  block_sum_store(acc, &partial[blockIdx.x]);
}

// band-pair output: fixed-point totals to FP64, times the normalisation and sign
__global__ void __launch_bounds__(kThreads) k_pairs_out(const unsigned long long *__restrict__ pairs, int n,
                                                         double scale, double *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = scale * ((double)(long long)pairs[i] / kPairScale);
}

// ---------------------------------------------------------------- reduction
constexpr int kRedThreads = 1024;
__global__ void __launch_bounds__(kRedThreads) k_reduce(const double *__restrict__ partial, int nblocks, int nw,
                                                         double scale, const double *__restrict__ dos, int ndos,
                                                         const double *__restrict__ omega,
                                                         const double *__restrict__ extra,
                                                         double *__restrict__ out) {
  const int k = blockIdx.x;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0, sd = 0.0;
  int b = threadIdx.x;
  for (; b + 3 * kRedThreads < nblocks; b += 4 * kRedThreads) {  // independent loads in flight
    s0 += partial[(long long)b * nw + k];
    s1 += partial[(long long)(b + kRedThreads) * nw + k];
    s2 += partial[(long long)(b + 2 * kRedThreads) * nw + k];
    s3 += partial[(long long)(b + 3 * kRedThreads) * nw + k];
  }
  for (; b < nblocks; b += kRedThreads) s0 += partial[(long long)b * nw + k];
  const bool add_dos = dos && (omega == nullptr || omega[k] == 0.0);
  if (add_dos)
    for (int i = threadIdx.x; i < ndos; i += kRedThreads) sd += dos[i];
  double v = ((s0 + s1) + (s2 + s3)) + sd;
  __shared__ double red[kRedThreads / 32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = red[threadIdx.x];
    v = warp_sum(v);
    if (threadIdx.x == 0) out[k] = scale * (extra ? v + extra[k] : v);
  }
}

}  // namespace

// ======================================================================= launchers
int static_blocks() { return kStaticBlocks; }

__global__ void __launch_bounds__(kThreads) k_c128_to_c64(const double2 *__restrict__ in, float2 *__restrict__ out,
                                                         long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double2 v = in[i];
    out[i] = make_float2((float)v.x, (float)v.y);
  }
}

cudaError_t launch_c128_to_c64(const void *in, void *out, long long n, cudaStream_t s) {
  k_c128_to_c64<<<device_sms() * 8, kThreads, 0, s>>>((const double2 *)in, (float2 *)out, n);
  return cudaGetLastError();
}

cudaError_t launch_overlap(const Grid &g, const double *, const void *C, int dtype, const Q &q, void *W2,
                           int fp64, cudaStream_t s, const void *C32) {
  const int w = q.hi - q.lo;
  const long long total = g.nc * (long long)w * w;
  long long nb = (total + kThreads - 1) / kThreads;
  const int blocks = (int)(nb < device_sms() * 16 ? nb : device_sms() * 16);
  if (blocks <= 0) return cudaSuccess;
  const bool small = (long long)g.norb * w <= kOvlSmall && !fp64;
  if (small) {
    // k side in complex64 (the plan's copy when the inputs are complex128)
    const float2 *Ck = (const float2 *)(C32 ? C32 : C);
    long long nbw = (g.nc + kWarps - 1) / kWarps;
    const int bw = (int)(nbw < device_sms() * 8 ? nbw : device_sms() * 8);
    if (q.Cq && dtype == DT_C128)
      k_overlap_small<float2, double2, float><<<bw, kThreads, 0, s>>>(g, Ck, (const double2 *)q.Cq, 1, q,
                                                                      (float *)W2);
    else if (q.Cq)
      k_overlap_small<float2, float2, float><<<bw, kThreads, 0, s>>>(g, Ck, (const float2 *)q.Cq, 1, q,
                                                                     (float *)W2);
    else
      k_overlap_small<float2, float2, float><<<bw, kThreads, 0, s>>>(g, Ck, Ck, 0, q, (float *)W2);
    return cudaGetLastError();
  }
  if (dtype == DT_C128) {
    const double2 *Cx = (const double2 *)C, *Cq = (const double2 *)q.Cq;
    if (fp64) k_overlap<double2, double><<<blocks, kThreads, 0, s>>>(g, Cx, Cq, q, (double *)W2);
    else k_overlap<double2, float><<<blocks, kThreads, 0, s>>>(g, Cx, Cq, q, (float *)W2);
  } else {
    const float2 *Cx = (const float2 *)C, *Cq = (const float2 *)q.Cq;
    if (fp64) k_overlap<float2, double><<<blocks, kThreads, 0, s>>>(g, Cx, Cq, q, (double *)W2);
    else k_overlap<float2, float><<<blocks, kThreads, 0, s>>>(g, Cx, Cq, q, (float *)W2);
  }
  return cudaGetLastError();
}

cudaError_t launch_bands(const double *E, long long nc, int nb, double ef, short *occ, short *emp, float *E32,
                         cudaStream_t s, float *E32lo) {
  long long nb_ = (nc + kThreads - 1) / kThreads;
  const int blocks = (int)(nb_ < device_sms() * 8 ? nb_ : device_sms() * 8);
  k_bands<<<blocks, kThreads, 0, s>>>(E, nc, nb, ef, occ, emp, E32, E32lo);
  return cudaGetLastError();
}

int device_sms() {
  int dev = 0, sms = kSMs;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

int static_max_ctas_per_sm(int fp64, int variant) {
  int nb = 0;
  cudaError_t e;
  if (fp64) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_static<true, 256, 1>, 256, 0);
  else if (variant == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_static<false, 128, 3>, 128, 0);
  else if (variant == 2) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_static<false, 256, 1>, 256, 0);
  else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_static<false, 256, 2>, 256, 0);
  return (e != cudaSuccess || nb < 1) ? 1 : nb;
}

int static_variants(int fp64) { return fp64 ? 1 : 3; }
int static_variant_threads(int fp64, int variant) { return !fp64 && variant == 1 ? 128 : 256; }

int static_persistent_blocks(int fp64) { return static_max_ctas_per_sm(fp64, 0) * device_sms(); }

long long static_batches(long long ntet) { return (ntet + 31) / 32; }
int static_tab_cap() { return kTabCap; }
size_t static_piece_bytes(int fp64) { return fp64 ? sizeof(Piece<double>) : sizeof(Piece<float>); }

cudaError_t launch_static(const Grid &g, const Tet &tet, const void *Ek, const void *Ekq, const Q &q,
                          const void *W2, int cma, int fp64, float tau, const short *occ, const short *empq,
                          const StaticBufs &sb, int nblocks, unsigned long long *counters, cudaStream_t s,
                          int variant) {
  cudaError_t e = cudaMemsetAsync(sb.next, 0, sizeof(int), s);  // batch counter
  if (e != cudaSuccess) return e;
  const long long nbatch = static_batches(g.ntet);
  if (fp64)
    k_static<true, 256, 1><<<nblocks, 256, 0, s>>>(g, tet, Ek, Ekq, q, W2, cma, tau, occ, empq, sb, counters);
  else if (variant == 1)
    k_static<false, 128, 3><<<nblocks, 128, 0, s>>>(g, tet, Ek, Ekq, q, W2, cma, tau, occ, empq, sb, counters);
  else if (variant == 2)
    k_static<false, 256, 1><<<nblocks, 256, 0, s>>>(g, tet, Ek, Ekq, q, W2, cma, tau, occ, empq, sb, counters);
  else
    k_static<false, 256, 2><<<nblocks, 256, 0, s>>>(g, tet, Ek, Ekq, q, W2, cma, tau, occ, empq, sb, counters);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  long long tb = (nbatch * 32 + kThreads - 1) / kThreads;
  const int tblocks = (int)(tb < device_sms() * 16 ? tb : device_sms() * 16);
  if (sb.off && sb.vals) {  // compacted queue
    k_tab_scan<<<1, 1024, 0, s>>>(sb.tq_n, nbatch, sb.off);
    if (fp64) k_tab_eval<true><<<device_sms() * 8, kThreads, 0, s>>>(nbatch, sb);
    else k_tab_eval<false><<<device_sms() * 8, kThreads, 0, s>>>(nbatch, sb);
    k_tab_sum<<<tblocks, kThreads, 0, s>>>(nbatch, sb);
  } else if (fp64) {
    k_static_tab<true><<<tblocks, kThreads, 0, s>>>(nbatch, sb);
  } else {
    k_static_tab<false><<<tblocks, kThreads, 0, s>>>(nbatch, sb);
  }
  return cudaGetLastError();
}

cudaError_t launch_dos(const Grid &g, const Tet &tet, const double *E, int lo, int hi, double *partial,
                       int nblocks, cudaStream_t s, unsigned long long *pairs) {
  k_dos<<<nblocks, kThreads, 0, s>>>(g, tet, E, lo, hi, partial, pairs);
  return cudaGetLastError();
}

cudaError_t launch_pairs_out(const unsigned long long *pairs, int n, double scale, double *out, cudaStream_t s) {
  k_pairs_out<<<(n + kThreads - 1) / kThreads, kThreads, 0, s>>>(pairs, n, scale, out);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const double *partial, int nblocks, int nw, double scale, const double *dos,
                          int ndos, const double *omega, double *out, cudaStream_t s, const double *extra) {
  k_reduce<<<nw, kRedThreads, 0, s>>>(partial, nblocks, nw, scale, dos, ndos, omega, extra, out);
  return cudaGetLastError();
}

}  // namespace chi0int
