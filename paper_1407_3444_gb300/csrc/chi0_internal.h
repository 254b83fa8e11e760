// chi0_internal.h -- interface between the C-ABI layer and the kernel translation unit.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace chi0int {

// n / d for 32-bit unsigned n by a multiply-high and shifts (Granlund-Montgomery): no
// integer-division sequence and no int<->float conversions in the index arithmetic.
struct FastDiv {
  unsigned d, m, s;
};
inline FastDiv make_fastdiv(unsigned d) {
  FastDiv f{d, 0u, 0u};
  if (d <= 1) return f;
  unsigned l = 0;
  while ((1ull << l) < d) ++l;                                   // l = ceil(log2 d)
  f.m = (unsigned)((((1ull << l) - d) << 32) / d + 1);           // floor(2^32 (2^l - d)/d) + 1
  f.s = l - 1;
  return f;
}
#ifdef __CUDACC__
__device__ __forceinline__ unsigned fdiv(unsigned n, const FastDiv &f) {
  if (f.d <= 1) return n;
  const unsigned t = __umulhi(n, f.m);
  return (t + ((n - t) >> 1)) >> f.s;
}
#endif

struct Grid {
  int n[3];   // cubes per axis
  int N[3];   // corners per axis
  int periodic;
  int nb, norb;
  long long nc;    // corners (< 2^31, checked when the plan is built)
  long long ntet;  // tetrahedra (< 2^31)
  double ef;
  FastDiv fn1, fn2;  // cube index decode: n1, n2
  FastDiv fN1, fN2;  // corner index decode: N1, N2
};

struct Tet {
  const int4 *corners;  // device [ntet] or nullptr (builtin mesh)
  const double *vol;    // device [ntet] or nullptr
  double vol_builtin;   // 1/(6 n0 n1 n2)
};

// one q point as the kernels see it
struct Q {
  const double *Eq;  // device [nc][nb] explicit energies at k+q, or nullptr (shift)
  const void *Cq;    // device [nc][norb][nb] explicit eigenvectors at k+q, or nullptr
  int shift[3];
  int lo, hi;        // band window
  int gamma;
};

enum { DT_C64 = 1, DT_C128 = 2 };

// |M_mn|^2 at every k corner for one q: W2[c][m-lo][n-lo] (fp64: double, else float)
cudaError_t launch_overlap(const Grid &g, const double *E, const void *C, int dtype, const Q &q,
                           void *W2, int fp64, cudaStream_t s, const void *C32);
// complex128 -> complex64 copy (the k-side eigenvectors of a mixed-precision plan)
cudaError_t launch_c128_to_c64(const void *in, void *out, long long n, cudaStream_t s);

// band bounds per corner: occ[c] (1 + highest occupied band), emp[c] (lowest empty band);
// E32 (optional) receives (float)(E - ef); E32lo (optional) the remainder
// (float)((E - ef) - E32), so that E32 + E32lo carries E - ef to ~2^-48 relative
cudaError_t launch_bands(const double *E, long long nc, int nb, double ef, short *occ, short *emp, float *E32,
                         cudaStream_t s, float *E32lo = nullptr);

// Work buffers of the static kernels (device memory owned by the plan).
struct StaticBufs {
  void *tq;        // queued final tetrahedra: [nbatch][static_tab_cap()] pieces
  int *tq_n;       // [nbatch] queued per batch
  double *partial; // [2 * nbatch]: series part, queued part
  int *next;       // batch counter
  int tcap;        // queue entries per batch (at most static_tab_cap())
  unsigned long long *pairs = nullptr;  // band-pair output: [w][w] fixed-point totals (or none)
  int *off = nullptr;      // compacted queue: [nbatch + 1] offsets and [nbatch * tcap] values
  double *vals = nullptr;  // (both null: one warp per batch walks its queue)
};

// static weights for one q: partial[2 * nbatch] (sum them for chi0); Ek/Ekq are the absolute
// FP64 energies (fp64) or the FP32 energies relative to eF (mixed); occ from the k
// energies, empq from the k+q energies
cudaError_t launch_static(const Grid &g, const Tet &tet, const void *Ek, const void *Ekq, const Q &q,
                          const void *W2, int cma, int fp64, float tau, const short *occ, const short *empq,
                          const StaticBufs &sb, int nblocks, unsigned long long *counters, cudaStream_t s, int variant = 0);
int static_persistent_blocks(int fp64);
long long static_batches(long long ntet);
int static_tab_cap();

// message of the last failed call made without a plan (chi0_last_error(NULL))
void set_global_error(const char *msg);
size_t static_piece_bytes(int fp64);

// Work buffers of the dynamic weights: one partial per (batch of 32 tetrahedra, frequency) for
// the pieces evaluated directly, and the far-field box moments (per warp, then summed)
struct DynBufs {
  double *partR, *partI;  // [nbatch][nw]
  void *box_tab;          // box centres and radii of the pass (dynamic_box_tab_bytes())
  double *box_part;       // [warps of the launch][dynamic_box_slots(fp64)] (FP32 kernel: int64 per CTA)
  double *box_tot;        // [dynamic_box_slots(fp64)]
  double *far;            // [nw]: Re contribution of the box multipoles per frequency
  void *fb;               // [warps of the launch][dynamic_fb_bytes(fp64)]: near-field entries
                          // left to the per-vertex table (scratch)
  unsigned long long *fx;   // FP32 kernel: [CTAs of the launch][2][dynamic_max_nw()] fixed-point sums
  unsigned long long *ctr;  // FP32 kernel: batch counter (reset by the launch)
};

// dynamic weights for one q and nw <= dynamic_max_nw() frequencies: partR/partI in *rows rows
// of nw (FP64: one per batch; FP32: one) and far[nw] (add far to the sum of partR)
cudaError_t launch_dynamic(const Grid &g, const Tet &tet, const void *Ek, const void *Ekq, const Q &q,
                           const void *W2, int cma, int fp64, float tau, const short *occ, const short *empq,
                           const double *omega, int nw, const DynBufs &db, int nblocks,
                           unsigned long long *counters, cudaStream_t s, const float *Eklo,
                           const float *Ekqlo, int *rows);
size_t dynamic_fx_bytes(int nblocks);
// Im only, for the Kramers-Kronig route: partI in *rows rows of nw (omega ascending, >= 0)
cudaError_t launch_dynamic_im(const Grid &g, const Tet &tet, const void *Ek, const void *Ekq, const Q &q,
                              const void *W2, int cma, int fp64, float tau, const short *occ, const short *empq,
                              const double *omega, int nw, const DynBufs &db, int nblocks,
                              unsigned long long *counters, cudaStream_t s, const float *Eklo,
                              const float *Ekqlo, int *rows);
// energies and eigenvectors at k+q (fractional q) by linear interpolation from the periodic
// mesh (chi0_interp.cu): Eq [nc][nb], Cq [nc][norb][nb] (C == nullptr: energies only), c64:
// complex64 vectors, else complex128
cudaError_t launch_interp_kq(const Grid &g, const double *E, const void *C, int c64, const double q[3], double *Eq,
                             void *Cq, cudaStream_t s);
// Re from Im (Kramers-Kronig, chi0_kk.cu): im[0..m) on u_j = j du (im[0] = 0, im = 0 from u_m on),
// re[i] at u_i, i < m, plus scale * (sum of dos[0..ndos)) at u = 0 when dos != NULL
cudaError_t launch_kk(const double *im, int m, double du, double scale, const double *dos, int ndos, double *re,
                      cudaStream_t s);
int dynamic_persistent_blocks(int fp64);
int dynamic_warps_per_cta(int fp64);
size_t dynamic_box_slots(int fp64);
size_t dynamic_box_tab_bytes();
size_t dynamic_fb_bytes(int fp64);
cudaError_t dynamic_prepare();  // kernel attributes (shared memory); call outside stream capture

// Gamma: intraband q -> 0 limit, tetrahedron DOS at eF: partial[nblocks]
cudaError_t launch_dos(const Grid &g, const Tet &tet, const double *E, int lo, int hi, double *partial,
                       int nblocks, cudaStream_t s, unsigned long long *pairs = nullptr);
// band-pair output: out[i] = scale * pairs[i] in FP64 (pairs: fixed-point totals of the static kernels)
cudaError_t launch_pairs_out(const unsigned long long *pairs, int n, double scale, double *out, cudaStream_t s);

// out[k] = scale * (sum_b partial[b*nw + k] (+ sum dos where omega == 0) (+ extra[k]))
cudaError_t launch_reduce(const double *partial, int nblocks, int nw, double scale, const double *dos,
                          int ndos, const double *omega, double *out, cudaStream_t s,
                          const double *extra = nullptr);

int static_blocks();
int dynamic_max_nw();

// |M_mn|^2 on the tensor cores (mixed precision): k side from the plan's complex64 copy C32,
// k+q side from q.Cq (complex64 or complex128, explicit) or C32 at the shifted corner.
// W2[c][m-lo][n-lo] FP32.  budget: clock cycles a bounded wait may take (<= 0: 2^31);
// test_stall: issue no MMA, so that the first wait runs out (error-path test).  A wait that
// runs out sets *err to 1.
enum { TC_TF32 = 0, TC_BF16X3 = 1, TC_BF16X6 = 2 };
constexpr size_t kTcSmemMax = 227 * 1024;
size_t overlap_tc_smem(int w, int norb, int mode);  // bytes of shared memory ((size_t)-1: w > 128)
int overlap_tc_max_corners(int w, int norb, int mode);  // corners per MMA round, untuned
// gcap > 0: at most gcap corners per MMA round (autotuner candidates)
cudaError_t launch_overlap_tc(const Grid &g, const void *C32, int dtype, const Q &q, float *W2, int mode,
                              long long budget, int test_stall, int gcap, int *err, cudaStream_t s);
// tensor-core throughput (TFLOP/s) of `iters` back-to-back MMAs per SM, M = 128, N = 256
cudaError_t tc_peak(int mode, int iters, double *tflops, double *ms);
// resident CTAs per SM of the weight kernels (occupancy limit) and SMs of the device
int static_max_ctas_per_sm(int fp64, int variant);
int static_variants(int fp64);                      // block shapes of the static weight kernel
int static_variant_threads(int fp64, int variant);  // threads per block of a shape
int dynamic_max_ctas_per_sm(int fp64);
int device_sms();

#ifdef __CUDACC__
// corner index with periodic wrap (32-bit: the plan checks that the mesh has fewer than 2^31
// corners), and the corner at integer offset s from corner c
__device__ __forceinline__ int wrap_idx(int i, int N) { return i >= N ? i - N : i; }
__device__ __forceinline__ long long cid(const Grid &g, int i0, int i1, int i2) {
  if (g.periodic) {
    i0 = wrap_idx(i0, g.N[0]);
    i1 = wrap_idx(i1, g.N[1]);
    i2 = wrap_idx(i2, g.N[2]);
  }
  return (long long)(unsigned)((i0 * g.N[1] + i1) * g.N[2] + i2);
}
__device__ __forceinline__ long long shift_corner(const Grid &g, long long c, const int s[3]) {
  const unsigned cu = (unsigned)c;
  const unsigned r = fdiv(cu, g.fN2);
  const int i2 = (int)(cu - r * (unsigned)g.N[2]);
  const unsigned i0 = fdiv(r, g.fN1);
  const int i1 = (int)(r - i0 * (unsigned)g.N[1]);
  return cid(g, (int)i0 + s[0], i1 + s[1], i2 + s[2]);
}
#endif

}  // namespace chi0int
