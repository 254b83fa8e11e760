// chi0_noalloc.cu -- chi0_static_noalloc: static chi0 with every work buffer in one
// file-scope device array instead of cudaMalloc'd memory.
//
// For callers that cannot allocate device memory at the point where they need chi0:
// cudaMalloc and cudaFree can synchronize the whole device and take unbounded time,
// which a real-time loop or a step inside a latency budget cannot afford, and some host
// applications hand all device memory to their own pool allocator, which must account
// for every byte and does not tolerate raw allocations beside it.  Such callers keep
// their inputs and outputs in memory they already own and let this entry point use the
// fixed scratch array below.
//
// The array (CHI0_NOALLOC_SCRATCH_BYTES) is part of the library image: every GPU that
// loads the library holds it until the process exits.  Host code cannot use the array's
// name as a device address; its address is looked up with cudaGetSymbolAddress once per
// device, the first time the entry point runs on that device (with the device current).
// All calls share the array and it keeps the previous call's contents, so everything that
// must start at zero is cleared on the caller's stream; two calls that overlap on the GPU
// (different streams, or different host threads on one device) race on it.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "../../include/chi0.h"
#include "chi0_internal.h"

using namespace chi0int;

static __device__ __align__(256) unsigned char g_chi0_scratch[CHI0_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
constexpr int kNoallocTabCap = 16;  // queue entries per batch (overflow is evaluated in place)
unsigned char *g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

int err(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  set_global_error(buf);
  return code;
}

// device address of the scratch array on the current device (looked up once per device)
int scratch_base(unsigned char **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return err(CHI0_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return err(CHI0_ENOTSUP, "device %d beyond %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_chi0_scratch);
    if (e != cudaSuccess || !p)
      return err(CHI0_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    g_scratch_ptr[dev] = (unsigned char *)p;
  }
  *out = g_scratch_ptr[dev];
  return CHI0_OK;
}

constexpr size_t kSat = ~(size_t)0;  // saturated size: larger than any scratch array

// a * b and a + b rounded up to 256, saturating at kSat instead of wrapping around
size_t mul_sat(size_t a, size_t b) { return (b != 0 && a > kSat / b) ? kSat : a * b; }
size_t align256(size_t x) { return x > kSat - 255 ? kSat : (x + 255) & ~(size_t)255; }

struct Layout {
  size_t occ, emp, occq, empq, E32, Eq32, C32, W2, next, counters, tq, tq_n, part, dos, total;
};

Layout layout(const Grid &g, int w, int fp64, int cma, int dtype) {
  Layout L{};
  // every size saturates instead of wrapping, so a mesh too large for the array can never
  // come out small here (total == kSat then fails the size check)
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align256(bytes > kSat - o ? kSat : o + bytes);
    return at;
  };
  const size_t nc = (size_t)g.nc, nb = (size_t)g.nb, no = (size_t)g.norb, ww = (size_t)w;
  const size_t nbatch = (size_t)static_batches(g.ntet);
  L.occ = take(mul_sat(sizeof(short), nc));
  L.emp = take(mul_sat(sizeof(short), nc));
  L.occq = take(mul_sat(sizeof(short), nc));
  L.empq = take(mul_sat(sizeof(short), nc));
  L.E32 = take(fp64 ? 0 : mul_sat(mul_sat(sizeof(float), nc), nb));
  L.Eq32 = take(fp64 ? 0 : mul_sat(mul_sat(sizeof(float), nc), nb));
  L.C32 = take((!fp64 && !cma && dtype == CHI0_C128) ? mul_sat(mul_sat(mul_sat(8, nc), no), nb) : 0);
  L.W2 = take(cma ? 0 : mul_sat(mul_sat(mul_sat(fp64 ? 8 : 4, nc), ww), ww));
  L.next = take(sizeof(int));
  L.counters = take(4 * sizeof(unsigned long long));
  L.tq = take(mul_sat(mul_sat(static_piece_bytes(fp64), nbatch), kNoallocTabCap));
  L.tq_n = take(mul_sat(sizeof(int), nbatch));
  L.part = take(mul_sat(sizeof(double), mul_sat(2, nbatch)));
  L.dos = take(mul_sat(sizeof(double), (size_t)static_blocks()));
  L.total = o;
  return L;
}

}  // namespace

extern "C" int chi0_static_noalloc(const chi0_kgrid_t *kg, chi0_band_window_t win, const chi0_opts_t *opts,
                                   const chi0_q_t *qs, int nq, double *chi) {
  if (!kg || !opts || !qs || !chi || nq <= 0) return err(CHI0_EINVAL, "NULL argument or nq <= 0");
  const chi0_opts_t &op = *opts;
  if (op.precision != CHI0_PREC_FP64 && op.precision != CHI0_PREC_MIXED)
    return err(CHI0_EINVAL, "precision %d unknown", op.precision);
  if (op.overlap != CHI0_OVL_FP32) return err(CHI0_ENOTSUP, "only the FP32 overlap mode is available here");
  for (int d = 0; d < 3; ++d)
    if (kg->n[d] < 1 || kg->n[d] > (1 << 12)) return err(CHI0_EINVAL, "n[%d] = %d out of range", d, kg->n[d]);
  if (kg->nbands < 1 || kg->nbands > 4096) return err(CHI0_EINVAL, "nbands = %d out of range", kg->nbands);
  if (!kg->energies) return err(CHI0_EINVAL, "energies is NULL");
  if (!op.cma && (!kg->evecs || kg->norb < 1 || (kg->evec_dtype != CHI0_C64 && kg->evec_dtype != CHI0_C128)))
    return err(CHI0_EINVAL, "eigenvectors (norb, dtype) required without CMA");
  if (!op.cma && kg->norb > 65536) return err(CHI0_EINVAL, "norb = %d out of range", kg->norb);
  if (win.lo < 0 || win.hi > kg->nbands || win.lo >= win.hi)
    return err(CHI0_EINVAL, "band window [%d, %d) outside [0, %d)", win.lo, win.hi, kg->nbands);
  const int fp64 = op.precision == CHI0_PREC_FP64;
  Grid g{};
  for (int d = 0; d < 3; ++d) {
    g.n[d] = kg->n[d];
    g.N[d] = kg->periodic ? kg->n[d] : kg->n[d] + 1;
  }
  g.periodic = kg->periodic ? 1 : 0;
  g.nb = kg->nbands;
  g.norb = op.cma ? 0 : kg->norb;
  g.nc = (long long)g.N[0] * g.N[1] * g.N[2];
  g.ntet = 6LL * g.n[0] * g.n[1] * g.n[2];
  g.ef = kg->e_fermi;
  g.fn1 = make_fastdiv((unsigned)g.n[1]);
  g.fn2 = make_fastdiv((unsigned)g.n[2]);
  g.fN1 = make_fastdiv((unsigned)g.N[1]);
  g.fN2 = make_fastdiv((unsigned)g.N[2]);
  if (g.nc >= (1LL << 31) || g.ntet >= (1LL << 31)) return err(CHI0_EINVAL, "mesh too large");
  const int dtype = op.cma ? CHI0_C128 : kg->evec_dtype;
  const int w = win.hi - win.lo;
  const long long nbatch = static_batches(g.ntet);
  const Layout L = layout(g, w, fp64, op.cma, dtype);
  if (L.total > (size_t)CHI0_NOALLOC_SCRATCH_BYTES)
    return err(CHI0_EINVAL, "this mesh needs %zu bytes of scratch; chi0_static_noalloc has %zu", L.total,
               (size_t)CHI0_NOALLOC_SCRATCH_BYTES);
  // q descriptors: windows and shifts (device pointers are the caller's)
  for (int iq = 0; iq < nq; ++iq) {
    const chi0_q_t &qd = qs[iq];
    const int lo = qd.win.lo < 0 ? win.lo : qd.win.lo, hi = qd.win.lo < 0 ? win.hi : qd.win.hi;
    if (lo < win.lo || hi > win.hi || lo >= hi) return err(CHI0_EINVAL, "q %d window outside the window", iq);
    if (qd.e_kq && !op.cma && !qd.c_kq) return err(CHI0_EINVAL, "q %d: e_kq without c_kq", iq);
    if (!qd.e_kq && !g.periodic) return err(CHI0_EINVAL, "q %d: on-grid shift needs a periodic grid", iq);
  }

  unsigned char *base = nullptr;
  int rc = scratch_base(&base);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)op.stream;
  short *occ = (short *)(base + L.occ), *emp = (short *)(base + L.emp);
  short *occq = (short *)(base + L.occq), *empq = (short *)(base + L.empq);
  float *E32 = fp64 ? nullptr : (float *)(base + L.E32), *Eq32 = fp64 ? nullptr : (float *)(base + L.Eq32);
  void *C32 = (!fp64 && !op.cma && dtype == CHI0_C128) ? (void *)(base + L.C32) : nullptr;
  void *W2 = op.cma ? nullptr : (void *)(base + L.W2);
  int *next = (int *)(base + L.next);
  unsigned long long *counters = (unsigned long long *)(base + L.counters);
  double *part = (double *)(base + L.part), *dos = (double *)(base + L.dos);
  StaticBufs sb{base + L.tq, (int *)(base + L.tq_n), part, next, kNoallocTabCap};
  Tet tet{nullptr, nullptr, 1.0 / (6.0 * g.n[0] * g.n[1] * g.n[2])};
  const double scale = op.sign == CHI0_SIGN_PAPER ? -2.0 : 2.0;
  cudaError_t e;
#define NA_CK(call)                                                                                  \
  do {                                                                                               \
    if ((e = (call)) != cudaSuccess) return err(CHI0_ECUDA, "%s: %s", #call, cudaGetErrorString(e)); \
  } while (0)
  NA_CK(cudaMemsetAsync(counters, 0, 4 * sizeof(unsigned long long), s));
  NA_CK(launch_bands(kg->energies, g.nc, g.nb, g.ef, occ, emp, E32, s));
  if (C32) NA_CK(launch_c128_to_c64(kg->evecs, C32, g.nc * (long long)g.norb * g.nb, s));
  const int grid = static_persistent_blocks(fp64);
  for (int iq = 0; iq < nq; ++iq) {
    const chi0_q_t &qd = qs[iq];
    Q q{};
    q.lo = qd.win.lo < 0 ? win.lo : qd.win.lo;
    q.hi = qd.win.lo < 0 ? win.hi : qd.win.hi;
    q.gamma = qd.gamma ? 1 : 0;
    bool zero = true;
    if (qd.e_kq) {
      q.Eq = qd.e_kq;
      q.Cq = qd.c_kq;
    } else {
      for (int d = 0; d < 3; ++d) {
        int v = qd.shift[d] % g.N[d];
        if (v < 0) v += g.N[d];
        q.shift[d] = v;
        zero = zero && v == 0;
      }
      if (zero) q.gamma = 1;
    }
    if (!op.cma) NA_CK(launch_overlap(g, kg->energies, kg->evecs, dtype, q, W2, fp64, s, C32));
    if (q.gamma) NA_CK(launch_dos(g, tet, kg->energies, q.lo, q.hi, dos, static_blocks(), s));
    const short *empq_use = emp;
    const void *Ek = fp64 ? (const void *)kg->energies : (const void *)E32, *Ekq = Ek;
    if (q.Eq) {
      NA_CK(launch_bands(q.Eq, g.nc, g.nb, g.ef, occq, empq, fp64 ? nullptr : Eq32, s));
      empq_use = empq;
      Ekq = fp64 ? (const void *)q.Eq : (const void *)Eq32;
    }
    NA_CK(launch_static(g, tet, Ek, Ekq, q, W2, op.cma, fp64, (float)op.tau, occ, empq_use, sb, grid, counters, s));
    NA_CK(launch_reduce(part, (int)(2 * nbatch), 1, scale, q.gamma ? dos : nullptr, static_blocks(), nullptr,
                        chi + iq, s));
  }
#undef NA_CK
  return CHI0_OK;
}
