// chi0_abi.cu -- the C-ABI of include/chi0.h: plan objects, validation, uploads and the
// per-q launch sequence overlap -> weights -> (Gamma DOS) -> reduction on one stream.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <stdint.h>
#include <vector>

#include "../../include/chi0.h"
#include "chi0_internal.h"

using namespace chi0int;

struct chi0_plan {
  Grid g;
  Tet tet;
  chi0_opts_t opts;
  chi0_band_window_t win;
  cudaStream_t stream;
  int dtype;
  double *E_d = nullptr;
  void *C_d = nullptr;
  bool own_E = false, own_C = false;
  int4 *tet_d = nullptr;
  double *vol_d = nullptr;
  void *W2_d = nullptr;
  double *partR = nullptr, *partI = nullptr, *dos_d = nullptr;
  double *out_d = nullptr;
  size_t out_cap = 0;
  double *omega_d = nullptr;
  size_t omega_cap = 0;
  double *Eq_stage = nullptr;                 // explicit k+q data from the host: two staging
  void *Cq_stage = nullptr;                   // buffers, filled on a copy stream while the
  double *Eq_stage2 = nullptr;                // previous q computes
  void *Cq_stage2 = nullptr;
  cudaStream_t copy_s = nullptr;
  cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
  int stage_slot = 0;
  double *E_alt = nullptr;                    // chi0_plan_stage: the second set of eigen-data
  void *C_alt = nullptr;                      // buffers, filled on a stream of its own while
  cudaStream_t next_s = nullptr;              // the plan's stream computes.  npend staged sets
  cudaEvent_t ev_staged[2] = {nullptr, nullptr};  // wait for calls (the oldest in the alt set,
  cudaEvent_t ev_readers = nullptr;           // a second one in the current set, which no call
  int npend = 0;                              // reads again); ev_staged: their copies done
  unsigned long long *counters_d = nullptr;
  short *occ_d = nullptr, *emp_d = nullptr, *occq_d = nullptr, *empq_d = nullptr;
  float *E32_d = nullptr, *Eq32_d = nullptr;  // energies - eF in FP32 (mixed precision): hi, then lo
  void *C32_d = nullptr;                      // complex64 copy of complex128 eigenvectors (mixed)
  int *next_d = nullptr;                      // [2] batch counter, FP64 list size
  int *err_d = nullptr;                       // error word of the bounded device waits
  cudaStream_t cap_s = nullptr;               // graph mode: private stream the graph runs on,
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;  // ordered after / before the plan's stream
  cudaGraph_t graph = nullptr;                // graph mode: the captured call and its key
  cudaGraphExec_t gexec = nullptr;
  std::vector<unsigned char> gkey;
  long long gkernels = 0;
  void *box_tab_d = nullptr;                  // dynamic weights: box table of the pass,
  double *box_part_d = nullptr;               // per-warp box moments, their totals and the
  double *box_tot_d = nullptr;                // boxes' share of Re per frequency
  double *far_d = nullptr;
  void *fb_d = nullptr;                       // dynamic weights: per-warp fallback entries,
  unsigned long long *fx_d = nullptr;         // per-CTA fixed-point sums (FP32) and the
  unsigned long long *ctr_d = nullptr;        // batch counter
  unsigned long long *pairs_fx_d = nullptr;   // band-pair output: fixed-point totals of one q,
  size_t pairs_fx_cap = 0;                    // and the FP64 results of the call (host outputs)
  double *pairs_out_d = nullptr;
  size_t pairs_out_cap = 0;
  double *ikq_E_d = nullptr;                  // chi0_interpolate_kq with host outputs
  void *ikq_C_d = nullptr;
  size_t ikq_E_cap = 0, ikq_C_cap = 0;
  void *tq_d = nullptr;                       // queued final tetrahedra per batch
  int *tq_n_d = nullptr;
  int *tq_off_d = nullptr;                    // compacted queue: offsets and values
  double *tq_val_d = nullptr;
  int static_grid = 0, dynamic_grid = 0;  // persistent CTAs of the weight kernels
  int static_variant = 0;                  // block shape of the static weight kernel
  int tc_gcap = 0;                         // corners per tensor-core round (0: most that fit)
  size_t part_cap = 0;
  chi0_stats_t stats;
  char err[512];
};

static char g_plan_err[512] = "";
static void drop_graph(chi0_plan_t *p);

namespace chi0int {
void set_global_error(const char *msg) { snprintf(g_plan_err, sizeof(g_plan_err), "%s", msg); }
}  // namespace chi0int

static int fail(chi0_plan_t *p, int code, const char *fmt, ...) {
  char *dst = p ? p->err : g_plan_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 512, fmt, ap);
  va_end(ap);
  return code;
}

#define CK(p, call)                                                                          \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return fail((p), e_ == cudaErrorMemoryAllocation ? CHI0_ENOMEM : CHI0_ECUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                        \
  } while (0)

static size_t cplx_size(int dtype) { return dtype == CHI0_C64 ? 8 : 16; }

// tensor-core precision form of a CHI0_OVL_* mode (not CHI0_OVL_FP32)
static int tc_mode(int overlap) {
  return overlap == CHI0_OVL_TF32 ? TC_TF32 : (overlap == CHI0_OVL_BF16X3 ? TC_BF16X3 : TC_BF16X6);
}

extern "C" void chi0_opts_default(chi0_opts_t *o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->precision = CHI0_PREC_FP64;
  o->overlap = CHI0_OVL_FP32;
  o->cma = 0;
  o->sign = CHI0_SIGN_POSITIVE;
  o->tau = 9.5367431640625e-7; /* 2^-20 */
  o->inputs_on_device = 0;
  o->outputs_on_device = 0;
  o->stream = nullptr;
  o->profile = 0;
  o->wait_budget = 0;
}

extern "C" int chi0_version(void) { return 106; }

extern "C" const char *chi0_last_error(const chi0_plan_t *p) { return p ? p->err : g_plan_err; }

extern "C" int chi0_plan_stats(const chi0_plan_t *p, chi0_stats_t *s) {
  if (!p || !s) return CHI0_EINVAL;
  *s = p->stats;
  return CHI0_OK;
}

static void release(chi0_plan_t *p) {
  if (!p) return;
  if (p->next_s) cudaStreamSynchronize(p->next_s);  // staged copies may still write either set
  drop_graph(p);
  if (p->own_E) cudaFree(p->E_d);
  if (p->own_C) cudaFree(p->C_d);
  cudaFree(p->tet_d);
  cudaFree(p->vol_d);
  cudaFree(p->W2_d);
  cudaFree(p->partR);
  cudaFree(p->partI);
  cudaFree(p->dos_d);
  cudaFree(p->out_d);
  cudaFree(p->omega_d);
  cudaFree(p->Eq_stage);
  cudaFree(p->Cq_stage);
  cudaFree(p->Eq_stage2);
  cudaFree(p->Cq_stage2);
  for (int i = 0; i < 2; ++i) {
    if (p->ev_copied[i]) cudaEventDestroy(p->ev_copied[i]);
    if (p->ev_free[i]) cudaEventDestroy(p->ev_free[i]);
  }
  if (p->copy_s) cudaStreamDestroy(p->copy_s);
  if (p->next_s) cudaStreamDestroy(p->next_s);
  cudaFree(p->E_alt);
  cudaFree(p->C_alt);
  for (int i = 0; i < 2; ++i)
    if (p->ev_staged[i]) cudaEventDestroy(p->ev_staged[i]);
  if (p->ev_readers) cudaEventDestroy(p->ev_readers);
  cudaFree(p->counters_d);
  cudaFree(p->occ_d);
  cudaFree(p->emp_d);
  cudaFree(p->empq_d);
  cudaFree(p->occq_d);
  cudaFree(p->E32_d);
  cudaFree(p->C32_d);
  cudaFree(p->Eq32_d);
  cudaFree(p->next_d);
  cudaFree(p->err_d);
  cudaFree(p->tq_d);
  cudaFree(p->tq_n_d);
  cudaFree(p->tq_off_d);
  cudaFree(p->tq_val_d);
  cudaFree(p->box_tab_d);
  cudaFree(p->box_part_d);
  cudaFree(p->box_tot_d);
  cudaFree(p->far_d);
  cudaFree(p->fb_d);
  cudaFree(p->fx_d);
  cudaFree(p->ctr_d);
  cudaFree(p->pairs_fx_d);
  cudaFree(p->pairs_out_d);
  cudaFree(p->ikq_E_d);
  cudaFree(p->ikq_C_d);
}

extern "C" void chi0_destroy(chi0_plan_t *p) {
  if (!p) return;
  if (p->stream) cudaStreamSynchronize(p->stream);
  else cudaDeviceSynchronize();
  release(p);
  delete p;
}

static int build_plan(chi0_plan_t *p, const chi0_kgrid_t *kg, const chi0_tetra_t *tt, chi0_band_window_t win,
                      const chi0_opts_t *o) {
  if (!kg) return fail(p, CHI0_EINVAL, "kgrid is NULL");
  if (o) p->opts = *o;
  else chi0_opts_default(&p->opts);
  const chi0_opts_t &op = p->opts;
  if (op.precision != CHI0_PREC_FP64 && op.precision != CHI0_PREC_MIXED)
    return fail(p, CHI0_EINVAL, "precision %d unknown", op.precision);
  if (op.overlap != CHI0_OVL_FP32 && op.overlap != CHI0_OVL_BF16X3 && op.overlap != CHI0_OVL_TF32 &&
      op.overlap != CHI0_OVL_BF16X6)
    return fail(p, CHI0_EINVAL, "overlap mode %d unknown", op.overlap);
  if (op.overlap != CHI0_OVL_FP32 && op.precision != CHI0_PREC_MIXED)
    return fail(p, CHI0_ENOTSUP, "tensor-core overlaps belong to the mixed-precision form");
  if (op.test_stall && op.overlap == CHI0_OVL_FP32)
    return fail(p, CHI0_EINVAL, "test_stall needs a tensor-core overlap mode");
  if (op.graph && op.test_stall) return fail(p, CHI0_EINVAL, "graph mode and test_stall exclude each other");
  if (!(op.tau >= 0.0 && op.tau < 1.0)) return fail(p, CHI0_EINVAL, "tau must lie in [0, 1)");
  for (int d = 0; d < 3; ++d)
    if (kg->n[d] < 1 || kg->n[d] > (1 << 12)) return fail(p, CHI0_EINVAL, "n[%d] = %d out of range", d, kg->n[d]);
  if (kg->nbands < 1 || kg->nbands > 4096) return fail(p, CHI0_EINVAL, "nbands = %d out of range", kg->nbands);
  if (!op.cma && (kg->norb < 1 || kg->norb > 65536)) return fail(p, CHI0_EINVAL, "norb = %d out of range", kg->norb);
  if (!kg->energies) return fail(p, CHI0_EINVAL, "energies is NULL");
  if (!op.cma && !kg->evecs) return fail(p, CHI0_EINVAL, "evecs is NULL without CMA");
  if (!op.cma && kg->evec_dtype != CHI0_C64 && kg->evec_dtype != CHI0_C128)
    return fail(p, CHI0_EINVAL, "evec_dtype %d unknown", kg->evec_dtype);
  if (win.lo < 0 || win.hi > kg->nbands || win.lo >= win.hi)
    return fail(p, CHI0_EINVAL, "band window [%d, %d) outside [0, %d)", win.lo, win.hi, kg->nbands);
  if (!(kg->e_fermi == kg->e_fermi)) return fail(p, CHI0_EINVAL, "e_fermi is NaN");

  Grid &g = p->g;
  for (int d = 0; d < 3; ++d) {
    g.n[d] = kg->n[d];
    g.N[d] = kg->periodic ? kg->n[d] : kg->n[d] + 1;
  }
  g.periodic = kg->periodic ? 1 : 0;
  g.nb = kg->nbands;
  g.norb = op.cma ? 0 : kg->norb;
  g.nc = (long long)g.N[0] * g.N[1] * g.N[2];
  g.ef = kg->e_fermi;
  p->win = win;
  p->dtype = op.cma ? CHI0_C128 : kg->evec_dtype;
  p->stream = (cudaStream_t)op.stream;

  // tetrahedra
  if (tt && tt->corners) {
    if (tt->ntet < 1 || !tt->volume) return fail(p, CHI0_EINVAL, "custom tetrahedra need ntet >= 1 and volumes");
    for (long long t = 0; t < tt->ntet; ++t)
      for (int i = 0; i < 4; ++i) {
        const long long c = tt->corners[4 * t + i];
        if (c < 0 || c >= g.nc) return fail(p, CHI0_EINVAL, "tetrahedron %lld corner %lld outside [0, %lld)", t, c, g.nc);
      }
    g.ntet = tt->ntet;
    CK(p, cudaMalloc(&p->tet_d, sizeof(int4) * g.ntet));
    CK(p, cudaMalloc(&p->vol_d, sizeof(double) * g.ntet));
    CK(p, cudaMemcpyAsync(p->tet_d, tt->corners, sizeof(int4) * g.ntet, cudaMemcpyHostToDevice, p->stream));
    CK(p, cudaMemcpyAsync(p->vol_d, tt->volume, sizeof(double) * g.ntet, cudaMemcpyHostToDevice, p->stream));
  } else {
    g.ntet = 6LL * g.n[0] * g.n[1] * g.n[2];
  }
  p->tet.corners = p->tet_d;
  p->tet.vol = p->vol_d;
  p->tet.vol_builtin = 1.0 / (6.0 * g.n[0] * g.n[1] * g.n[2]);

  // eigen-data
  const size_t eb = sizeof(double) * (size_t)g.nc * g.nb;
  const size_t cb = op.cma ? 0 : cplx_size(p->dtype) * (size_t)g.nc * g.norb * g.nb;
  if (op.inputs_on_device) {
    p->E_d = (double *)kg->energies;
    p->C_d = (void *)kg->evecs;
  } else {
    for (long long c = 0; c < g.nc; ++c)
      for (int b = 1; b < g.nb; ++b)
        if (kg->energies[c * g.nb + b] < kg->energies[c * g.nb + b - 1])
          return fail(p, CHI0_EINVAL, "energies not ascending at corner %lld band %d", c, b);
    CK(p, cudaMalloc(&p->E_d, eb));
    p->own_E = true;
    CK(p, cudaMemcpyAsync(p->E_d, kg->energies, eb, cudaMemcpyHostToDevice, p->stream));
    if (!op.cma) {
      CK(p, cudaMalloc(&p->C_d, cb));
      p->own_C = true;
      CK(p, cudaMemcpyAsync(p->C_d, kg->evecs, cb, cudaMemcpyHostToDevice, p->stream));
    }
  }
  // scratch: |M|^2 at the plan's window, block partials, counters
  const int w = win.hi - win.lo;
  if (op.overlap != CHI0_OVL_FP32 && !op.cma &&
      overlap_tc_smem(w, g.norb, tc_mode(op.overlap)) > kTcSmemMax)
    return fail(p, CHI0_ENOTSUP, "tensor-core overlaps: a band window of %d with %d orbitals exceeds one tile", w,
                g.norb);
  CK(p, cudaMalloc(&p->err_d, sizeof(int)));
  CK(p, cudaMemsetAsync(p->err_d, 0, sizeof(int), p->stream));
  if (!op.cma) {
    const size_t es = op.precision == CHI0_PREC_FP64 ? sizeof(double) : sizeof(float);
    CK(p, cudaMalloc(&p->W2_d, es * (size_t)g.nc * w * w));
  }
  const size_t np = (size_t)static_batches(g.ntet) * dynamic_max_nw();
  size_t ns = 2 * (size_t)static_batches(g.ntet);
  if (ns < (size_t)static_blocks()) ns = (size_t)static_blocks();
  p->part_cap = np > ns ? np : ns;
  CK(p, cudaMalloc(&p->partR, sizeof(double) * p->part_cap));
  CK(p, cudaMalloc(&p->partI, sizeof(double) * p->part_cap));
  CK(p, cudaMalloc(&p->dos_d, sizeof(double) * static_blocks()));
  CK(p, cudaMalloc(&p->counters_d, sizeof(unsigned long long) * 4));
  if (g.nc >= (1LL << 31)) return fail(p, CHI0_EINVAL, "more than 2^31 corners");
  CK(p, cudaMalloc(&p->occ_d, sizeof(short) * g.nc));
  CK(p, cudaMalloc(&p->emp_d, sizeof(short) * g.nc));
  CK(p, cudaMalloc(&p->empq_d, sizeof(short) * g.nc));
  CK(p, cudaMalloc(&p->occq_d, sizeof(short) * g.nc));
  CK(p, cudaMalloc(&p->next_d, 2 * sizeof(int)));
  {
    const long long nbatch = static_batches(g.ntet);
    const int fp64 = op.precision == CHI0_PREC_FP64;
    CK(p, cudaMalloc(&p->tq_d, static_piece_bytes(fp64) * (size_t)nbatch * static_tab_cap()));
    CK(p, cudaMalloc(&p->tq_n_d, sizeof(int) * (size_t)nbatch));
    CK(p, cudaMalloc(&p->tq_off_d, sizeof(int) * (size_t)(nbatch + 1)));
    CK(p, cudaMalloc(&p->tq_val_d, sizeof(double) * (size_t)nbatch * static_tab_cap()));
  }
  if (op.precision == CHI0_PREC_MIXED) {
    CK(p, cudaMalloc(&p->E32_d, 2 * sizeof(float) * (size_t)g.nc * g.nb));
    CK(p, cudaMalloc(&p->Eq32_d, 2 * sizeof(float) * (size_t)g.nc * g.nb));
  }
  CK(p, launch_bands(p->E_d, g.nc, g.nb, g.ef, p->occ_d, p->emp_d, p->E32_d, p->stream,
                     p->E32_d ? p->E32_d + (size_t)g.nc * g.nb : nullptr));
  if (op.precision == CHI0_PREC_MIXED && !op.cma && p->dtype == CHI0_C128) {
    const long long ne = g.nc * (long long)g.norb * g.nb;
    CK(p, cudaMalloc(&p->C32_d, 8 * (size_t)ne));
    CK(p, launch_c128_to_c64(p->C_d, p->C32_d, ne, p->stream));
  }
  g.fn1 = make_fastdiv((unsigned)g.n[1]);
  g.fn2 = make_fastdiv((unsigned)g.n[2]);
  g.fN1 = make_fastdiv((unsigned)g.N[1]);
  g.fN2 = make_fastdiv((unsigned)g.N[2]);
  if (g.ntet >= (1LL << 31)) return fail(p, CHI0_EINVAL, "more than 2^31 tetrahedra");
  p->static_grid = static_persistent_blocks(op.precision == CHI0_PREC_FP64);
  CK(p, dynamic_prepare());
  p->dynamic_grid = dynamic_persistent_blocks(op.precision == CHI0_PREC_FP64);
  {
    // dynamic weights: box moments of every warp of the largest grid the autotuner may pick
    const int fp64 = op.precision == CHI0_PREC_FP64;
    const size_t warps = (size_t)dynamic_max_ctas_per_sm(fp64) * device_sms() * dynamic_warps_per_cta(fp64);
    CK(p, cudaMalloc(&p->box_tab_d, dynamic_box_tab_bytes()));
    CK(p, cudaMalloc(&p->box_part_d, sizeof(double) * warps * dynamic_box_slots(fp64)));
    CK(p, cudaMalloc(&p->box_tot_d, sizeof(double) * dynamic_box_slots(fp64)));
    CK(p, cudaMalloc(&p->far_d, sizeof(double) * dynamic_max_nw()));
    CK(p, cudaMalloc(&p->fb_d, warps * dynamic_fb_bytes(fp64)));
    CK(p, cudaMalloc(&p->fx_d, dynamic_fx_bytes(dynamic_max_ctas_per_sm(fp64) * device_sms())));
    CK(p, cudaMalloc(&p->ctr_d, sizeof(unsigned long long)));
  }
  CK(p, cudaMemsetAsync(p->counters_d, 0, sizeof(unsigned long long) * 4, p->stream));
  CK(p, cudaStreamSynchronize(p->stream));
  memset(&p->stats, 0, sizeof(p->stats));
  return CHI0_OK;
}

extern "C" int chi0_plan(const chi0_kgrid_t *kg, const chi0_tetra_t *tt, chi0_band_window_t win,
                         const chi0_opts_t *o, chi0_plan_t **out) {
  if (!out) return fail(nullptr, CHI0_EINVAL, "out is NULL");
  *out = nullptr;
  chi0_plan_t *p = new (std::nothrow) chi0_plan_t();
  if (!p) return fail(nullptr, CHI0_ENOMEM, "host allocation failed");
  p->err[0] = 0;
  int rc = build_plan(p, kg, tt, win, o);
  if (rc != CHI0_OK) {
    snprintf(g_plan_err, sizeof(g_plan_err), "%s", p->err);
    release(p);
    delete p;
    return rc;
  }
  *out = p;
  return CHI0_OK;
}

// ------------------------------------------------------------------ per-call helpers
namespace {

struct Timer {
  chi0_plan_t *p;
  std::vector<cudaEvent_t> ev;
  std::vector<int> kind;
  bool on = true;  // off while a graph is being captured
  int start(int k) {
    if (!p->opts.profile || !on) return 0;
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return -1;
    ev.push_back(a);
    ev.push_back(b);
    kind.push_back(k);
    return cudaEventRecord(a, p->stream) == cudaSuccess ? 0 : -1;
  }
  int stop() {
    if (!p->opts.profile || !on) return 0;
    return cudaEventRecord(ev.back(), p->stream) == cudaSuccess ? 0 : -1;
  }
  void collect() {
    for (size_t i = 0; i < kind.size(); ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]) == cudaSuccess) {
        p->stats.time_ms[kind[i]] += ms;
        p->stats.launches[kind[i]] += 1;
      }
    }
    for (auto e : ev) cudaEventDestroy(e);
    ev.clear();
    kind.clear();
  }
};

int ensure(chi0_plan_t *p, void **buf, size_t *cap, size_t bytes) {
  if (*cap >= bytes) return CHI0_OK;
  cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  CK(p, cudaMalloc(buf, bytes));
  *cap = bytes;
  return CHI0_OK;
}

// Resolves one q descriptor into device pointers (staging host explicit data).
// the checks of one q descriptor (every q of a call is checked before its first launch)
int validate_q(chi0_plan_t *p, const chi0_q_t &qd) {
  const int lo = qd.win.lo < 0 ? p->win.lo : qd.win.lo, hi = qd.win.lo < 0 ? p->win.hi : qd.win.hi;
  if (lo < p->win.lo || hi > p->win.hi || lo >= hi)
    return fail(p, CHI0_EINVAL, "q window [%d, %d) outside the plan window [%d, %d)", lo, hi, p->win.lo, p->win.hi);
  if (qd.e_kq && !p->opts.cma && !qd.c_kq) return fail(p, CHI0_EINVAL, "explicit e_kq needs c_kq without CMA");
  if (!qd.e_kq && !p->g.periodic) return fail(p, CHI0_EINVAL, "on-grid q shift needs a periodic grid");
  return CHI0_OK;
}

int prepare_q(chi0_plan_t *p, const chi0_q_t &qd, Q &q, int *slot_used) {
  *slot_used = -1;
  const Grid &g = p->g;
  q.lo = qd.win.lo < 0 ? p->win.lo : qd.win.lo;
  q.hi = qd.win.lo < 0 ? p->win.hi : qd.win.hi;
  if (q.lo < p->win.lo || q.hi > p->win.hi || q.lo >= q.hi)
    return fail(p, CHI0_EINVAL, "q window [%d, %d) outside the plan window [%d, %d)", q.lo, q.hi, p->win.lo, p->win.hi);
  q.gamma = qd.gamma ? 1 : 0;
  q.Eq = nullptr;
  q.Cq = nullptr;
  if (qd.e_kq) {
    if (!p->opts.cma && !qd.c_kq) return fail(p, CHI0_EINVAL, "explicit e_kq needs c_kq without CMA");
    for (int d = 0; d < 3; ++d) q.shift[d] = 0;
    if (p->opts.inputs_on_device) {
      q.Eq = qd.e_kq;
      q.Cq = qd.c_kq;
    } else {
      // staging buffer `slot` (alternating): its copy waits until the q that used it last
      // is done, runs on the copy stream, and the compute stream waits for the copy, so the
      // copy of one q overlaps the kernels of the one before
      const int slot = p->stage_slot;
      p->stage_slot ^= 1;
      if (!p->copy_s) {
        CK(p, cudaStreamCreateWithFlags(&p->copy_s, cudaStreamNonBlocking));
        for (int i = 0; i < 2; ++i) {
          CK(p, cudaEventCreateWithFlags(&p->ev_copied[i], cudaEventDisableTiming));
          CK(p, cudaEventCreateWithFlags(&p->ev_free[i], cudaEventDisableTiming));
        }
      }
      double *&Eb = slot ? p->Eq_stage2 : p->Eq_stage;
      void *&Cb = slot ? p->Cq_stage2 : p->Cq_stage;
      const size_t eb = sizeof(double) * (size_t)g.nc * g.nb;
      if (!Eb) CK(p, cudaMalloc(&Eb, eb));
      CK(p, cudaStreamWaitEvent(p->copy_s, p->ev_free[slot], 0));
      CK(p, cudaMemcpyAsync(Eb, qd.e_kq, eb, cudaMemcpyHostToDevice, p->copy_s));
      q.Eq = Eb;
      if (!p->opts.cma) {
        const size_t cb = cplx_size(p->dtype) * (size_t)g.nc * g.norb * g.nb;
        if (!Cb) CK(p, cudaMalloc(&Cb, cb));
        CK(p, cudaMemcpyAsync(Cb, qd.c_kq, cb, cudaMemcpyHostToDevice, p->copy_s));
        q.Cq = Cb;
      }
      CK(p, cudaEventRecord(p->ev_copied[slot], p->copy_s));
      CK(p, cudaStreamWaitEvent(p->stream, p->ev_copied[slot], 0));
      *slot_used = slot;
    }
  } else {
    if (!g.periodic) return fail(p, CHI0_EINVAL, "on-grid q shift needs a periodic grid");
    bool zero = true;
    for (int d = 0; d < 3; ++d) {
      int s = qd.shift[d] % g.N[d];
      if (s < 0) s += g.N[d];
      q.shift[d] = s;
      zero = zero && s == 0;
    }
    if (zero) q.gamma = 1;
  }
  return CHI0_OK;
}

}  // namespace

// Every launch and device-side copy of one call, in stream order (the part a CUDA graph
// captures): counters, then per q the overlap, DOS, band bounds, weights and reductions.
static int enqueue_call(chi0_plan_t *p, const chi0_q_t *qs, int nq, const double *om_d, int nw, bool dyn,
                        double *outR, double *outI, Timer &tm, bool tc, double *outP = nullptr,
                        double kk_du = 0.0) {
  const chi0_opts_t &op = p->opts;
  const int fp64 = op.precision == CHI0_PREC_FP64;
  const double scale = op.sign == CHI0_SIGN_PAPER ? -2.0 : 2.0;
  cudaStream_t s = p->stream;
  CK(p, cudaMemsetAsync(p->counters_d, 0, sizeof(unsigned long long) * 4, s));
  size_t poff = 0;  // band-pair output: offset of this q's w x w block
  for (int iq = 0; iq < nq; ++iq) {
    Q q;
    int slot = -1;
    int rc = prepare_q(p, qs[iq], q, &slot);
    if (rc) return rc;
    const int wq = q.hi - q.lo;
    unsigned long long *pfx = outP ? p->pairs_fx_d : nullptr;
    if (pfx) CK(p, cudaMemsetAsync(pfx, 0, sizeof(unsigned long long) * wq * wq, s));
    if (!op.cma) {
      tm.start(CHI0_K_OVERLAP);
      if (tc)
        CK(p, launch_overlap_tc(p->g, p->C32_d ? p->C32_d : p->C_d, p->dtype, q, (float *)p->W2_d,
                                tc_mode(op.overlap), op.wait_budget, op.test_stall, p->tc_gcap,
                                p->err_d, s));
      else
        CK(p, launch_overlap(p->g, p->E_d, p->C_d, p->dtype, q, p->W2_d, fp64, s, p->C32_d));
      p->stats.kernels += 1;
      tm.stop();
    }
    const int ndos = static_blocks();
    if (q.gamma) {
      tm.start(CHI0_K_DOS);
      CK(p, launch_dos(p->g, p->tet, p->E_d, q.lo, q.hi, p->dos_d, ndos, s, pfx));
      p->stats.kernels += 1;
      tm.stop();
    }
    const int nb = (int)static_batches(p->g.ntet);
    const short *empq = p->emp_d;
    const void *Ek = fp64 ? (const void *)p->E_d : (const void *)p->E32_d;
    const void *Ekq = Ek;
    const size_t ncb = (size_t)p->g.nc * p->g.nb;
    const float *Eklo = fp64 ? nullptr : p->E32_d + ncb, *Ekqlo = Eklo;
    if (q.Eq) {
      tm.start(CHI0_K_BANDS);
      CK(p, launch_bands(q.Eq, p->g.nc, p->g.nb, p->g.ef, p->occq_d, p->empq_d, fp64 ? nullptr : p->Eq32_d, s,
                         fp64 ? nullptr : p->Eq32_d + ncb));
      p->stats.kernels += 1;
      tm.stop();
      empq = p->empq_d;
      Ekq = fp64 ? (const void *)q.Eq : (const void *)p->Eq32_d;
      if (!fp64) Ekqlo = p->Eq32_d + ncb;
    }
    if (!dyn) {
      // (the compacted queue indexes its pieces in 32 bits)
      const bool compact = (long long)nb * static_tab_cap() < (1LL << 31);
      StaticBufs sb{p->tq_d, p->tq_n_d, p->partR, p->next_d, static_tab_cap(), pfx,
                    compact ? p->tq_off_d : nullptr, compact ? p->tq_val_d : nullptr};
      tm.start(CHI0_K_STATIC);
      CK(p, launch_static(p->g, p->tet, Ek, Ekq, q, p->W2_d, op.cma, fp64, (float)op.tau, p->occ_d, empq, sb,
                          p->static_grid, p->counters_d, s, p->static_variant));
      p->stats.kernels += compact ? 4 : 2;
      tm.stop();
      tm.start(CHI0_K_REDUCE);
      CK(p, launch_reduce(p->partR, 2 * nb, 1, scale, q.gamma ? p->dos_d : nullptr, ndos, nullptr, outR + iq, s));
      p->stats.kernels += 1;
      if (pfx) {
        CK(p, launch_pairs_out(pfx, wq * wq, scale, outP + poff, s));
        p->stats.kernels += 1;
        poff += (size_t)wq * wq;
      }
      tm.stop();
    } else if (kk_du > 0.0) {
      // Kramers-Kronig route: Im alone on the uniform grid (passes of at most maxw nodes), then
      // Re from Im over the whole grid
      const int maxw = dynamic_max_nw();
      for (int w0 = 0; w0 < nw; w0 += maxw) {
        const int nwc = nw - w0 < maxw ? nw - w0 : maxw;
        DynBufs db{p->partR, p->partI, p->box_tab_d, p->box_part_d, p->box_tot_d, p->far_d, p->fb_d, p->fx_d,
                   p->ctr_d};
        int rows = nb;
        tm.start(CHI0_K_DYNAMIC);
        CK(p, launch_dynamic_im(p->g, p->tet, Ek, Ekq, q, p->W2_d, op.cma, fp64, (float)op.tau, p->occ_d, empq,
                                om_d + w0, nwc, db, p->dynamic_grid, p->counters_d, s, Eklo, Ekqlo, &rows));
        p->stats.kernels += fp64 ? 1 : 2;
        tm.stop();
        tm.start(CHI0_K_REDUCE);
        CK(p, launch_reduce(p->partI, rows, nwc, scale, nullptr, 0, nullptr, outI + (size_t)iq * nw + w0, s));
        p->stats.kernels += 1;
        tm.stop();
      }
      tm.start(CHI0_K_REDUCE);
      CK(p, launch_kk(outI + (size_t)iq * nw, nw, kk_du, scale, q.gamma ? p->dos_d : nullptr, ndos,
                      outR + (size_t)iq * nw, s));
      p->stats.kernels += 1;
      tm.stop();
    } else {
      const int maxw = dynamic_max_nw();
      for (int w0 = 0; w0 < nw; w0 += maxw) {
        const int nwc = nw - w0 < maxw ? nw - w0 : maxw;
        DynBufs db{p->partR, p->partI, p->box_tab_d, p->box_part_d, p->box_tot_d, p->far_d, p->fb_d, p->fx_d,
                   p->ctr_d};
        int rows = nb;
        tm.start(CHI0_K_DYNAMIC);
        CK(p, launch_dynamic(p->g, p->tet, Ek, Ekq, q, p->W2_d, op.cma, fp64, (float)op.tau, p->occ_d, empq,
                             om_d + w0, nwc, db, p->dynamic_grid, p->counters_d, s, Eklo, Ekqlo, &rows));
        p->stats.kernels += fp64 ? 4 : 5;  // box table, weights, box sums, box evaluation (+ row sums)
        tm.stop();
        tm.start(CHI0_K_REDUCE);
        CK(p, launch_reduce(p->partR, rows, nwc, scale, q.gamma ? p->dos_d : nullptr, ndos, om_d + w0,
                            outR + (size_t)iq * nw + w0, s, p->far_d));
        CK(p, launch_reduce(p->partI, rows, nwc, scale, nullptr, 0, nullptr, outI + (size_t)iq * nw + w0, s));
        p->stats.kernels += 2;
        tm.stop();
      }
    }
    if (slot >= 0) CK(p, cudaEventRecord(p->ev_free[slot], s));  // its staging buffer is free again
  }
  return CHI0_OK;
}

// graph key: everything the captured sequence depends on besides the plan itself
static std::vector<unsigned char> call_key(const chi0_q_t *qs, int nq, const double *om_d, int nw, bool dyn,
                                           const double *outR, const double *outI) {
  std::vector<unsigned char> k(sizeof(chi0_q_t) * (size_t)nq + 64, 0);
  memcpy(k.data(), qs, sizeof(chi0_q_t) * (size_t)nq);
  unsigned char *t = k.data() + sizeof(chi0_q_t) * (size_t)nq;
  const long long v[5] = {(long long)nq, (long long)nw, (long long)dyn, (long long)(uintptr_t)om_d,
                          (long long)(uintptr_t)outR};
  memcpy(t, v, sizeof(v));
  const long long w = (long long)(uintptr_t)outI;
  memcpy(t + sizeof(v), &w, sizeof(w));
  return k;
}

static void drop_graph(chi0_plan_t *p) {
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->cap_s) cudaStreamDestroy(p->cap_s);
  if (p->ev_in) cudaEventDestroy(p->ev_in);
  if (p->ev_out) cudaEventDestroy(p->ev_out);
  p->cap_s = nullptr;
  p->ev_in = p->ev_out = nullptr;
  p->gexec = nullptr;
  p->graph = nullptr;
  p->gkey.clear();
  p->gkernels = 0;
}

// band bounds and FP32 copies of the plan's current eigen-data (the mixed form's inputs)
static int derive_inputs(chi0_plan_t *p) {
  const Grid &g = p->g;
  CK(p, launch_bands(p->E_d, g.nc, g.nb, g.ef, p->occ_d, p->emp_d, p->E32_d, p->stream,
                     p->E32_d ? p->E32_d + (size_t)g.nc * g.nb : nullptr));
  p->stats.kernels += 1;
  if (p->C32_d) {
    CK(p, launch_c128_to_c64(p->C_d, p->C32_d, g.nc * (long long)g.norb * g.nb, p->stream));
    p->stats.kernels += 1;
  }
  return CHI0_OK;
}

// the oldest set staged by chi0_plan_stage (always in the alt buffers) becomes the current
// eigen-data: the plan's stream waits for its copies, and the sets swap places (a second
// staged set, in the old current buffers, is then the one in the alt buffers)
static int take_staged(chi0_plan_t *p) {
  if (p->npend == 0) return CHI0_OK;
  drop_graph(p);  // a captured call holds the old pointers
  CK(p, cudaStreamWaitEvent(p->stream, p->ev_staged[0], 0));
  double *e = p->E_d;
  p->E_d = p->E_alt;
  p->E_alt = e;
  void *c = p->C_d;
  p->C_d = p->C_alt;
  p->C_alt = c;
  cudaEvent_t ev = p->ev_staged[0];
  p->ev_staged[0] = p->ev_staged[1];
  p->ev_staged[1] = ev;
  p->npend -= 1;
  return derive_inputs(p);
}

static int run(chi0_plan_t *p, const chi0_q_t *qs, int nq, const double *omega, int nw, double *re,
               double *im, double *pairs = nullptr, double kk_du = 0.0) {
  if (!p) return fail(nullptr, CHI0_EINVAL, "plan is NULL");
  if (nq <= 0 || !qs) return fail(p, CHI0_EINVAL, "nq = %d or q NULL", nq);
  const bool dyn = omega != nullptr;
  if (dyn && (nw <= 0 || !re || !im)) return fail(p, CHI0_EINVAL, "dynamic call needs nw > 0, re and im");
  if (!dyn && !re) return fail(p, CHI0_EINVAL, "chi is NULL");
  for (int iq = 0; iq < nq; ++iq) {  // validation before any launch
    const int rc = validate_q(p, qs[iq]);
    if (rc) return rc;
  }
  {
    const int rc = take_staged(p);
    if (rc) return rc;
  }
  const chi0_opts_t &op = p->opts;
  const int fp64 = op.precision == CHI0_PREC_FP64;
  cudaStream_t s = p->stream;
  Timer tm{p, {}, {}};
  const int nwo = dyn ? nw : 1;
  const size_t outn = (size_t)nq * nwo * (dyn ? 2 : 1);
  double *outR = nullptr, *outI = nullptr;
  const double *om_d = nullptr;
  if (op.outputs_on_device) {
    outR = re;
    outI = dyn ? im : nullptr;
  } else {
    int rc = ensure(p, (void **)&p->out_d, &p->out_cap, sizeof(double) * outn);
    if (rc) return rc;
    outR = p->out_d;
    outI = dyn ? p->out_d + (size_t)nq * nw : nullptr;
  }
  if (dyn) {
    if (op.inputs_on_device || kk_du > 0.0) {  // (the Kramers-Kronig grid is already on the device)
      om_d = omega;
    } else {
      int rc = ensure(p, (void **)&p->omega_d, &p->omega_cap, sizeof(double) * nw);
      if (rc) return rc;
      CK(p, cudaMemcpyAsync(p->omega_d, omega, sizeof(double) * nw, cudaMemcpyHostToDevice, s));
      om_d = p->omega_d;
    }
  }
  const bool tc = op.overlap != CHI0_OVL_FP32 && !op.cma && !fp64;
  // band-pair output: fixed-point scratch for the widest window, and room for every q's block
  double *outP = nullptr;
  size_t npairs = 0;
  if (pairs) {
    const int wp = p->win.hi - p->win.lo;
    int rc = ensure(p, (void **)&p->pairs_fx_d, &p->pairs_fx_cap, sizeof(unsigned long long) * wp * wp);
    if (rc) return rc;
    for (int iq = 0; iq < nq; ++iq) {
      const int lo = qs[iq].win.lo < 0 ? p->win.lo : qs[iq].win.lo, hi = qs[iq].win.lo < 0 ? p->win.hi : qs[iq].win.hi;
      npairs += (size_t)(hi - lo) * (hi - lo);
    }
    if (op.outputs_on_device) {
      outP = pairs;
    } else {
      rc = ensure(p, (void **)&p->pairs_out_d, &p->pairs_out_cap, sizeof(double) * npairs);
      if (rc) return rc;
      outP = p->pairs_out_d;
    }
  }
  if (op.graph && !pairs && !(kk_du > 0.0)) {
    // replay the captured sequence when the call matches the one captured, else capture anew
    std::vector<unsigned char> key = call_key(qs, nq, om_d, nw, dyn, outR, outI);
    if (!p->gexec || key != p->gkey) {
      drop_graph(p);
      for (int iq = 0; iq < nq; ++iq)
        if ((qs[iq].e_kq || qs[iq].c_kq) && !op.inputs_on_device)
          return fail(p, CHI0_ENOTSUP, "graph mode needs device-resident inputs");
      // the graph is captured on (and later launched on) a private stream: the plan's stream
      // may be the legacy default stream, which cannot be captured
      CK(p, cudaStreamCreateWithFlags(&p->cap_s, cudaStreamNonBlocking));
      CK(p, cudaEventCreateWithFlags(&p->ev_in, cudaEventDisableTiming));
      CK(p, cudaEventCreateWithFlags(&p->ev_out, cudaEventDisableTiming));
      Timer off{p, {}, {}, false};
      const long long k0 = p->stats.kernels;
      CK(p, cudaStreamBeginCapture(p->cap_s, cudaStreamCaptureModeThreadLocal));
      p->stream = p->cap_s;
      const int rc = enqueue_call(p, qs, nq, om_d, nw, dyn, outR, outI, off, tc);
      p->stream = s;
      cudaGraph_t g = nullptr;
      const cudaError_t ec = cudaStreamEndCapture(p->cap_s, &g);
      if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
      }
      if (ec != cudaSuccess) return fail(p, CHI0_ECUDA, "graph capture: %s", cudaGetErrorString(ec));
      p->graph = g;
      const cudaError_t ei = cudaGraphInstantiate(&p->gexec, g, 0);
      if (ei != cudaSuccess) {
        drop_graph(p);
        return fail(p, CHI0_ECUDA, "graph instantiate: %s", cudaGetErrorString(ei));
      }
      p->gkey = key;
      p->gkernels = p->stats.kernels - k0;
      p->stats.kernels = k0;
    }
    tm.start(CHI0_K_GRAPH);
    CK(p, cudaEventRecord(p->ev_in, s));
    CK(p, cudaStreamWaitEvent(p->cap_s, p->ev_in, 0));
    CK(p, cudaGraphLaunch(p->gexec, p->cap_s));
    CK(p, cudaEventRecord(p->ev_out, p->cap_s));
    CK(p, cudaStreamWaitEvent(s, p->ev_out, 0));
    tm.stop();
    p->stats.kernels += p->gkernels;
  } else {
    const int rc = enqueue_call(p, qs, nq, om_d, nw, dyn, outR, outI, tm, tc, outP, kk_du);
    if (rc) return rc;
  }
  if (tc) {  // the tensor-core overlap's bounded waits report through the error word
    int herr = 0;
    CK(p, cudaMemcpyAsync(&herr, p->err_d, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(p, cudaStreamSynchronize(s));
    if (herr) {
      CK(p, cudaMemsetAsync(p->err_d, 0, sizeof(int), s));
      CK(p, cudaStreamSynchronize(s));
      return fail(p, CHI0_ETIMEOUT, "tensor-core overlap: a bounded wait ran out of its budget");
    }
  }
  if (!op.outputs_on_device) {
    CK(p, cudaMemcpyAsync(re, outR, sizeof(double) * nq * nwo, cudaMemcpyDeviceToHost, s));
    if (dyn) CK(p, cudaMemcpyAsync(im, outI, sizeof(double) * nq * nw, cudaMemcpyDeviceToHost, s));
    if (pairs) CK(p, cudaMemcpyAsync(pairs, outP, sizeof(double) * npairs, cudaMemcpyDeviceToHost, s));
  }
  if (op.profile || !op.outputs_on_device) CK(p, cudaStreamSynchronize(s));
  CK(p, cudaGetLastError());
  if (op.profile) {
    unsigned long long cnt[4] = {0, 0, 0, 0};
    CK(p, cudaMemcpy(cnt, p->counters_d, sizeof(cnt), cudaMemcpyDeviceToHost));
    p->stats.pieces += (long long)cnt[0];
    p->stats.fp64_evals += (long long)cnt[1];
    p->stats.queue_overflow += (long long)cnt[2];
    p->stats.box_pieces += (long long)cnt[3];
  }
  tm.collect();
  p->stats.calls += 1;
  return CHI0_OK;
}

extern "C" int chi0_static(chi0_plan_t *p, const chi0_q_t *q, int nq, double *chi) {
  return run(p, q, nq, nullptr, 0, chi, nullptr);
}

extern "C" int chi0_static_pairs(chi0_plan_t *p, const chi0_q_t *q, int nq, double *chi, double *pairs) {
  if (!pairs) return fail(p, CHI0_EINVAL, "pairs is NULL");
  if (p && p->win.hi - p->win.lo > 1024) return fail(p, CHI0_EINVAL, "band-pair output: window wider than 1024");
  return run(p, q, nq, nullptr, 0, chi, nullptr, pairs);
}

extern "C" int chi0_plan_update(chi0_plan_t *p, const double *energies, const void *evecs) {
  if (!p) return fail(nullptr, CHI0_EINVAL, "plan is NULL");
  if (!energies) return fail(p, CHI0_EINVAL, "energies is NULL");
  if (!p->opts.cma && !evecs) return fail(p, CHI0_EINVAL, "evecs is NULL without CMA");
  const Grid &g = p->g;
  const chi0_opts_t &op = p->opts;
  const size_t eb = sizeof(double) * (size_t)g.nc * g.nb;
  const size_t cb = op.cma ? 0 : cplx_size(p->dtype) * (size_t)g.nc * g.norb * g.nb;
  drop_graph(p);  // a captured call holds the old pointers
  if (p->npend > 0) {  // the new data replace staged sets, whose copies may still write the
    CK(p, cudaStreamWaitEvent(p->stream, p->ev_staged[p->npend - 1], 0));  // current buffers
    p->npend = 0;
  }
  if (op.inputs_on_device) {
    p->E_d = (double *)energies;
    if (!op.cma) p->C_d = (void *)evecs;
  } else {
    for (long long c = 0; c < g.nc; ++c)
      for (int b = 1; b < g.nb; ++b)
        if (energies[c * g.nb + b] < energies[c * g.nb + b - 1])
          return fail(p, CHI0_EINVAL, "energies not ascending at corner %lld band %d", c, b);
    CK(p, cudaMemcpyAsync(p->E_d, energies, eb, cudaMemcpyHostToDevice, p->stream));
    if (!op.cma) CK(p, cudaMemcpyAsync(p->C_d, evecs, cb, cudaMemcpyHostToDevice, p->stream));
  }
  const int rc = derive_inputs(p);
  if (rc) return rc;
  CK(p, cudaGetLastError());
  return CHI0_OK;
}

extern "C" int chi0_plan_stage(chi0_plan_t *p, const double *energies, const void *evecs) {
  if (!p) return fail(nullptr, CHI0_EINVAL, "plan is NULL");
  if (!energies) return fail(p, CHI0_EINVAL, "energies is NULL");
  if (!p->opts.cma && !evecs) return fail(p, CHI0_EINVAL, "evecs is NULL without CMA");
  if (p->opts.inputs_on_device) return fail(p, CHI0_EINVAL, "staging copies host inputs; a device-input plan adopts new pointers with chi0_plan_update");
  if (p->npend >= 2) return fail(p, CHI0_EINVAL, "two staged sets wait for calls already");
  const Grid &g = p->g;
  const size_t eb = sizeof(double) * (size_t)g.nc * g.nb;
  const size_t cb = p->opts.cma ? 0 : cplx_size(p->dtype) * (size_t)g.nc * g.norb * g.nb;
  for (long long c = 0; c < g.nc; ++c)
    for (int b = 1; b < g.nb; ++b)
      if (energies[c * g.nb + b] < energies[c * g.nb + b - 1])
        return fail(p, CHI0_EINVAL, "energies not ascending at corner %lld band %d", c, b);
  if (!p->next_s) {
    CK(p, cudaStreamCreateWithFlags(&p->next_s, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) CK(p, cudaEventCreateWithFlags(&p->ev_staged[i], cudaEventDisableTiming));
    CK(p, cudaEventCreateWithFlags(&p->ev_readers, cudaEventDisableTiming));
  }
  if (!p->E_alt) CK(p, cudaMalloc(&p->E_alt, eb));
  if (cb && !p->C_alt) CK(p, cudaMalloc(&p->C_alt, cb));
  // nothing staged: the copies go to the alt buffers; one set staged (in the alt buffers): to
  // the current ones, which the next call swaps out unread.  Either way the buffers' readers
  // are enqueued on the plan's stream before this point, so the copies wait for that work.
  double *E_dst = p->npend == 0 ? p->E_alt : p->E_d;
  void *C_dst = p->npend == 0 ? p->C_alt : p->C_d;
  CK(p, cudaEventRecord(p->ev_readers, p->stream));
  CK(p, cudaStreamWaitEvent(p->next_s, p->ev_readers, 0));
  CK(p, cudaMemcpyAsync(E_dst, energies, eb, cudaMemcpyHostToDevice, p->next_s));
  if (cb) CK(p, cudaMemcpyAsync(C_dst, evecs, cb, cudaMemcpyHostToDevice, p->next_s));
  CK(p, cudaEventRecord(p->ev_staged[p->npend], p->next_s));
  p->npend += 1;
  return CHI0_OK;
}

extern "C" int chi0_interpolate_kq(chi0_plan_t *p, const double *qfrac, double *e_kq, void *c_kq) {
  if (!p) return fail(nullptr, CHI0_EINVAL, "plan is NULL");
  if (!qfrac || !e_kq) return fail(p, CHI0_EINVAL, "qfrac or e_kq is NULL");
  if (!p->g.periodic) return fail(p, CHI0_EINVAL, "k+q interpolation needs a periodic grid");
  for (int d = 0; d < 3; ++d)
    if (!(fabs(qfrac[d]) < 1e6)) return fail(p, CHI0_EINVAL, "qfrac[%d] = %g", d, qfrac[d]);
  {
    const int rc = take_staged(p);
    if (rc) return rc;
  }
  const Grid &g = p->g;
  const bool vecs = c_kq && !p->opts.cma;
  const size_t eb = sizeof(double) * (size_t)g.nc * g.nb;
  const size_t cb = vecs ? cplx_size(p->dtype) * (size_t)g.nc * g.norb * g.nb : 0;
  double *Eo = e_kq;
  void *Co = vecs ? c_kq : nullptr;
  if (!p->opts.inputs_on_device) {  // host outputs: through device scratch
    int rc = ensure(p, (void **)&p->ikq_E_d, &p->ikq_E_cap, eb);
    if (rc) return rc;
    Eo = p->ikq_E_d;
    if (vecs) {
      rc = ensure(p, &p->ikq_C_d, &p->ikq_C_cap, cb);
      if (rc) return rc;
      Co = p->ikq_C_d;
    }
  }
  CK(p, launch_interp_kq(g, p->E_d, vecs ? p->C_d : nullptr, p->dtype == CHI0_C64, qfrac, Eo, Co, p->stream));
  p->stats.kernels += 1;
  if (!p->opts.inputs_on_device) {
    CK(p, cudaMemcpyAsync(e_kq, Eo, eb, cudaMemcpyDeviceToHost, p->stream));
    if (vecs) CK(p, cudaMemcpyAsync(c_kq, Co, cb, cudaMemcpyDeviceToHost, p->stream));
    CK(p, cudaStreamSynchronize(p->stream));
  }
  CK(p, cudaGetLastError());
  return CHI0_OK;
}

extern "C" int chi0_dynamic_kk(chi0_plan_t *p, const chi0_q_t *q, int nq, double wmax, int nkk, double *re,
                               double *im) {
  if (!p) return fail(nullptr, CHI0_EINVAL, "plan is NULL");
  if (!(wmax > 0.0) || !(wmax < 1e300) || nkk < 2) return fail(p, CHI0_EINVAL, "wmax = %g, nkk = %d", wmax, nkk);
  const double du = wmax / (nkk - 1);
  std::vector<double> grid((size_t)nkk);
  for (int j = 0; j < nkk; ++j) grid[(size_t)j] = j * du;
  int rc = ensure(p, (void **)&p->omega_d, &p->omega_cap, sizeof(double) * nkk);
  if (rc) return rc;
  CK(p, cudaMemcpyAsync(p->omega_d, grid.data(), sizeof(double) * nkk, cudaMemcpyHostToDevice, p->stream));
  CK(p, cudaStreamSynchronize(p->stream));  // (the host grid goes out of scope)
  return run(p, q, nq, p->omega_d, nkk, re, im, nullptr, du);
}

extern "C" int chi0_dynamic(chi0_plan_t *p, const chi0_q_t *q, int nq, const double *omega, int nw, double *re,
                            double *im) {
  if (!omega) return fail(p, CHI0_EINVAL, "omega is NULL");
  return run(p, q, nq, omega, nw, re, im);
}

// ---------------------------------------------------------------- autotuner
// Wall time of one call on the plan's stream (CUDA events; the call itself may synchronize).
static int timed_call(chi0_plan_t *p, const chi0_q_t *q, int nq, const double *omega, int nw, double *re,
                      double *im, float *ms) {
  cudaEvent_t a, b;
  CK(p, cudaEventCreate(&a));
  CK(p, cudaEventCreate(&b));
  CK(p, cudaEventRecord(a, p->stream));
  const int rc = run(p, q, nq, omega, nw, re, im);
  if (rc) {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return rc;
  }
  CK(p, cudaEventRecord(b, p->stream));
  CK(p, cudaEventSynchronize(b));
  CK(p, cudaEventElapsedTime(ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return CHI0_OK;
}

extern "C" int chi0_tune(chi0_plan_t *p, const chi0_q_t *q, int nq, const double *omega, int nw, double *re,
                         double *im, chi0_tune_t *res) {
  if (!p) return fail(nullptr, CHI0_EINVAL, "plan is NULL");
  if (!res) return fail(p, CHI0_EINVAL, "result is NULL");
  memset(res, 0, sizeof(*res));
  const chi0_opts_t &op = p->opts;
  const int fp64 = op.precision == CHI0_PREC_FP64;
  const bool dyn = omega != nullptr;
  const int sms = device_sms();
  const int graph = p->opts.graph;
  p->opts.graph = 0;  // every candidate runs its own launch sequence
  float ms = 0.f;
  int rc = run(p, q, nq, omega, nw, re, im);  // warm-up (first-touch, module load)
  if (!rc) rc = timed_call(p, q, nq, omega, nw, re, im, &ms);
  if (rc) {
    p->opts.graph = graph;
    return rc;
  }
  res->default_ms = ms;
  float best = ms;
  int cand = 1;
  // 1. block shape (static) and persistent CTAs per SM of the weight kernel this call uses
  int *grid = dyn ? &p->dynamic_grid : &p->static_grid;
  int best_grid = *grid, best_var = p->static_variant;
  const int nvar = dyn ? 1 : static_variants(fp64);
  for (int v = 0; v < nvar && !rc; ++v) {
    const int maxc = dyn ? dynamic_max_ctas_per_sm(fp64) : static_max_ctas_per_sm(fp64, v);
    for (int c = 1; c <= maxc; ++c) {
      if (c * sms == best_grid && (dyn || v == best_var)) continue;  // the untuned shape
      *grid = c * sms;
      if (!dyn) p->static_variant = v;
      rc = timed_call(p, q, nq, omega, nw, re, im, &ms);
      if (rc) break;
      ++cand;
      if (ms < best) {
        best = ms;
        best_grid = *grid;
        best_var = v;
      }
    }
  }
  *grid = best_grid;
  if (!dyn) p->static_variant = best_var;
  // 2. corners per tensor-core round (the tile's M/N packing)
  const bool tc = op.overlap != CHI0_OVL_FP32 && !op.cma && !fp64;
  int best_g = p->tc_gcap;
  if (!rc && tc) {
    const int gmax = overlap_tc_max_corners(p->win.hi - p->win.lo, p->g.norb, tc_mode(op.overlap));
    for (int gc = 1; gc <= gmax; gc = gc < 4 ? gc + 1 : gc * 2) {
      p->tc_gcap = gc;
      rc = timed_call(p, q, nq, omega, nw, re, im, &ms);
      if (rc) break;
      ++cand;
      if (ms < best) {
        best = ms;
        best_g = gc;
      }
    }
    p->tc_gcap = best_g;
  }
  p->opts.graph = graph;
  drop_graph(p);  // a graph captured before tuning holds the old launch shapes
  if (rc) return rc;
  res->static_variant = p->static_variant;
  res->static_threads = static_variant_threads(fp64, p->static_variant);
  res->static_ctas_per_sm = p->static_grid / sms;
  res->dynamic_ctas_per_sm = p->dynamic_grid / sms;
  res->tc_corners_per_round = p->tc_gcap;
  res->candidates = cand;
  res->best_ms = best;
  return CHI0_OK;
}
