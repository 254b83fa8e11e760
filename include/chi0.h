/*
 * chi0.h -- C-ABI of the GB300 (sm_103a) bare-susceptibility library.
 *
 * Computes the non-interacting susceptibility of Heil, Sormann, Boeri, Aichhorn and
 * von der Linden, "Accurate bare susceptibilities from full-potential ab initio
 * calculations" (Sec. II):
 *
 *   Re chi0(q,w) =  sum_{n,m} int_1BZ dk/(4 pi^3) Th(eF - e^m_k) Th(e^n_{k+q} - eF)
 *                   |<m,k|e^{-iq.r}|n,k+q>|^2 [1/(e^m_k - e^n_{k+q} + w) + 1/(e^m_k - e^n_{k+q} - w)]
 *                                                                                    (Eq. 1)
 *   Im chi0(q,w) = -sum_{n,m} int_1BZ dk/(4 pi^2) Th Th |<..>|^2 delta(w + e^m_k - e^n_{k+q})
 *                                                                         (Eq. 2, w >= 0)
 *   Im chi0(q,-w) = -Im chi0(q,w)                                                  (Eq. 3)
 *
 * by the linear tetrahedron method with the two carvings of Sec. II (first by
 * Th(eF - e^m_k), then by Th(e^n_{k+q} - eF), Eq. 4), energies and |M|^2 linearly
 * interpolated on every tetrahedron, and closed-form integrals on the final
 * tetrahedra (static w = 0, PV real part, delta-function imaginary part).
 *
 * Matrix elements use the tight-binding form M_mn(k,q) = sum_o conj(C_k[o][m]) C_{k+q}[o][n]
 * (Sec. III footnote; orbitals at the cell origin, periodic gauge), or |M|^2 = 1 (the
 * constant-matrix-element approximation, CMA, Sec. III).
 *
 * Units and normalisation: k is integrated in fractional coordinates (BZ volume 1);
 * chi0 is returned per unit cell, both spins, in states/(energy unit) -- i.e. the
 * dk/(4 pi^3) measure of Eq. 1 times the cell volume.  Energies in any unit (eV, Ha).
 *
 * Threading: a plan is used by one host thread at a time; all work of a plan is ordered on
 * the CUDA stream given in its options (host-to-device copies of staged eigen-data and of
 * explicit k+q data run on copy streams of the plan's own, ordered against that stream by
 * events).  Every call returns CHI0_OK (0) or a negative
 * status; no C++ exception crosses this interface.  Validation happens before any
 * launch.  After any error the plan can still be destroyed, and chi0_last_error()
 * describes the failure.
 */
#ifndef CHI0_H
#define CHI0_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
#define CHI0_OK 0
#define CHI0_EINVAL -1    /* invalid argument (sizes, window, pointers, layout)      */
#define CHI0_ENOMEM -2    /* device or host allocation failed                        */
#define CHI0_ECUDA -3     /* CUDA runtime error (launch, copy, device fault)         */
#define CHI0_ETIMEOUT -4  /* a bounded device-side wait ran out of its budget        */
#define CHI0_ENOTSUP -5   /* option combination not supported                        */
#define CHI0_EINTERNAL -6 /* internal consistency check failed                        */

/* ---------------------------------------------------------------- enumerations */
#define CHI0_C64 1  /* complex64: interleaved float (re, im)  */
#define CHI0_C128 2 /* complex128: interleaved double (re, im) */

#define CHI0_PREC_FP64 0  /* every step in FP64 (overlaps, weights, accumulation)          */
#define CHI0_PREC_MIXED 1 /* FP32 overlaps/weights, FP64 in the near-degenerate branches,
                             FP64 or exact 64-bit fixed-point accumulation                */

#define CHI0_OVL_FP32 0   /* mixed precision: overlaps with FP32 FMA on the CUDA cores     */
#define CHI0_OVL_BF16X3 1 /* mixed precision: overlaps on the tensor cores (tcgen05), each
                             operand split x = hi + lo into two BF16 pieces, products
                             hi*hi + hi*lo + lo*hi, FP32 accumulate (band window <= 128)  */
#define CHI0_OVL_TF32 2   /* mixed precision: overlaps on the tensor cores, one product of
                             round-to-nearest TF32 operands, FP32 accumulate (window
                             <= 128)                                                      */
#define CHI0_OVL_BF16X6 3 /* mixed precision: overlaps on the tensor cores, three-piece BF16
                             split x = p0 + p1 + p2, the six products pa*pb with a + b <= 2,
                             FP32 accumulate (band window <= 128; the tile must fit in
                             227 KB of shared memory: 3 (128 + 2w) (4 norb) bytes)        */

#define CHI0_SIGN_POSITIVE 0 /* return -(Eq. 1) and -(Eq. 2): static chi0 > 0, Im >= 0 (w>0) */
#define CHI0_SIGN_PAPER 1    /* return Eq. 1 and Eq. 2 exactly as printed                    */

/* ---------------------------------------------------------------- input structs */
/* k mesh and eigen-data at its corners.
 *   n[3]       cubes per reciprocal axis.
 *   periodic   1: Gamma-centred periodic grid, n0*n1*n2 corners at fractional k = i/n,
 *                 corner indices wrap modulo n (tight-binding models);
 *              0: open grid spanning one cube edge to edge, (n0+1)(n1+1)(n2+1) corners,
 *                 no wrap (free-electron tests); q must then be given explicitly.
 *   Corner index c = (i0*N1 + i1)*N2 + i2 with N the corner counts per axis.
 *   energies   [Nc][nbands] float64, ascending per corner.
 *   evecs      [Nc][norb][nbands] complex (evec_dtype): evecs[c][o][b] is the weight of
 *              orbital o in band b at corner c.  May be NULL only with opts.cma = 1.
 *   e_fermi    Fermi level (an input: the library never solves for it).
 * Host or device pointers according to opts.inputs_on_device. */
typedef struct {
  int n[3];
  int periodic;
  int nbands;
  int norb;
  const double *energies;
  const void *evecs;
  int evec_dtype;
  double e_fermi;
} chi0_kgrid_t;

/* Tetrahedral mesh (Sec. II: the integration domain split into tetrahedra).
 *   corners == NULL: builtin mesh, 6 tetrahedra per cube sharing the cube's
 *     (000)-(111) diagonal, tetrahedron 6*cube + p = {000, e_a, e_a + e_b, 111} for the
 *     p-th axis order (a, b, c) in lexicographic order of the permutations of (0,1,2);
 *     cube = (i0*n1 + i1)*n2 + i2; each of volume 1/(6 n0 n1 n2).
 *   corners != NULL: ntet tetrahedra, corners[4*t + i] corner indices, volume[t] their
 *     fractional volumes (BZ volume 1).  Always HOST pointers, copied by chi0_plan. */
typedef struct {
  int ntet;
  const int32_t *corners;
  const double *volume;
} chi0_tetra_t;

/* Band window [lo, hi): both the occupied band m and the empty band n run over it
 * (Sec. III band truncation). */
typedef struct {
  int lo, hi;
} chi0_band_window_t;

/* One q point.
 *   e_kq == NULL: on-grid q, k+q corner = corner shifted by shift[] (periodic grids).
 *   e_kq != NULL: explicit energies [Nc][nbands] at k+q for every corner c, and (unless
 *     CMA) c_kq [Nc][norb][nbands] eigenvectors at k+q (same layout/dtype as the plan).
 *     Host or device according to opts.inputs_on_device; read during the call only.
 *   win   per-q band window; {-1, -1} selects the plan's window.
 *   gamma 1: q is Gamma (or a reciprocal lattice vector).  Eq. 1 then has an empty
 *     intraband region; the library replaces the intraband terms by their q -> 0 limit,
 *     the density of states N(eF) (Sec. III), added to the static value and to Re at
 *     w = 0.  An all-zero shift with e_kq == NULL sets this automatically. */
typedef struct {
  int shift[3];
  const double *e_kq;
  const void *c_kq;
  chi0_band_window_t win;
  int gamma;
} chi0_q_t;

/* Options (initialise with chi0_opts_default).
 *   precision     CHI0_PREC_FP64 | CHI0_PREC_MIXED.
 *   overlap       CHI0_OVL_* (mixed precision only).
 *   cma           1: |M|^2 = 1 (no eigenvectors needed).
 *   sign          CHI0_SIGN_POSITIVE | CHI0_SIGN_PAPER.
 *   tau           mixed precision: knot-gap threshold (relative to the largest knot)
 *                 below which a final tetrahedron's weights are evaluated in FP64.
 *   inputs_on_device   1: every energy/eigenvector pointer (plan and q) is a device
 *                 pointer the caller keeps alive; 0: host pointers, copied.
 *   outputs_on_device  1: chi/re/im are device pointers; 0: host pointers.
 *   stream        cudaStream_t (NULL = legacy default stream) for every copy and launch.
 *   profile       1: time each kernel with CUDA events on the stream (chi0_plan_stats).
 *   wait_budget   clock cycles one bounded device-side wait may take before the call
 *                 fails with CHI0_ETIMEOUT (0 = 2^31, about one second).
 *   test_stall    error-path test hook: 1 makes the tensor-core overlap kernel issue no
 *                 MMA, so that its bounded wait runs out and the call returns
 *                 CHI0_ETIMEOUT; 0 in normal use.
 *   graph         1: each chi0_static / chi0_dynamic call's launches (every q, every
 *                 frequency pass) are captured once into a CUDA graph and replayed by later
 *                 calls with the same q descriptors, frequency and output pointers (a
 *                 different call is captured anew).  Explicit k+q data must then be device
 *                 pointers (inputs_on_device); with profile, time_ms[CHI0_K_GRAPH] holds the
 *                 graph launches. */
typedef struct {
  int precision;
  int overlap;
  int cma;
  int sign;
  double tau;
  int inputs_on_device;
  int outputs_on_device;
  void *stream;
  int profile;
  long long wait_budget;
  int test_stall;
  int graph;
  int reserved[6];
} chi0_opts_t;

typedef struct chi0_plan chi0_plan_t;

/* Per-kernel timing and work counters accumulated over a plan's calls (opts.profile):
 * time_ms[k] / launches[k] for k = CHI0_K_* (CUDA events on the plan's stream around each
 * launch), calls, and the final-tetrahedron and FP64-branch counts of the weight kernels. */
#define CHI0_K_OVERLAP 0
#define CHI0_K_STATIC 1
#define CHI0_K_DYNAMIC 2
#define CHI0_K_REDUCE 3
#define CHI0_K_DOS 4
#define CHI0_K_BANDS 5
#define CHI0_K_GRAPH 6 /* graph mode: one replay of a captured call */
#define CHI0_K_COUNT 8
typedef struct {
  double time_ms[CHI0_K_COUNT];
  long long launches[CHI0_K_COUNT];
  long long calls;
  long long pieces;     /* final tetrahedra evaluated (profile mode)                     */
  long long fp64_evals; /* weight evaluations taken by the FP64 branch (mixed, profile)  */
  long long kernels;    /* kernel launches made by the plan's calls (always counted)     */
  long long queue_overflow; /* static weights (profile): final tetrahedra that found their
                               batch's queue of long-series pieces full and were evaluated
                               in place by the carving warp instead                      */
  long long box_pieces;     /* dynamic weights (profile): final tetrahedra whose principal-
                               value terms were gathered into a box of D (far frequencies
                               by the box's moments) instead of evaluated per frequency    */
} chi0_stats_t;

/* ---------------------------------------------------------------- entry points */

/* Fills *opts with defaults: FP64, FP32 overlaps, exact |M|^2, positive sign,
 * tau = 2^-20, host inputs and outputs, default stream, no profiling. */
void chi0_opts_default(chi0_opts_t *opts);

/* Builds a plan for one k mesh (Sec. II: the tetrahedron decomposition and the corner
 * eigen-data).  Validates every size, copies host inputs (or adopts device pointers),
 * and allocates the device scratch for the largest window.  *out receives the plan
 * (NULL on error).  Errors: CHI0_EINVAL (bad sizes, window outside [0, nbands),
 * evecs missing without CMA, non-periodic grid with builtin tetrahedra missing),
 * CHI0_ENOMEM, CHI0_ECUDA. */
int chi0_plan(const chi0_kgrid_t *kgrid, const chi0_tetra_t *tetra, chi0_band_window_t window,
              const chi0_opts_t *opts, chi0_plan_t **out);

/* New eigen-data for an existing plan: the same mesh, bands, orbitals, eigenvector type and
 * Fermi level, new energies [Nk][nbands] (ascending per k) and eigenvectors [Nk][norb][nbands]
 * (ignored with CMA).  Host inputs are checked and their copies into the plan's buffers
 * enqueued on the plan's stream (the arrays must stay unchanged until the stream has passed
 * the copies); device inputs are adopted (the caller keeps them alive).  The band bounds and the FP32 copies of the mixed form
 * are rebuilt, a captured graph is dropped.  Lets repeated calls on new data reuse the plan's
 * allocations.  Errors: CHI0_EINVAL (NULL plan or energies, evecs NULL without CMA, energies
 * not ascending), CHI0_ECUDA. */
int chi0_plan_update(chi0_plan_t *plan, const double *energies, const void *evecs);

/* Staged eigen-data for a later call, for plans with host inputs: the arrays (same shapes and
 * rules as chi0_plan_update) are checked and their copies enqueued on a copy stream of the
 * plan's own, and the call returns.  Up to two staged sets wait for calls; each call that
 * reads the eigen-data (chi0_static, chi0_static_pairs, chi0_dynamic, chi0_dynamic_kk,
 * chi0_interpolate_kq, chi0_tune) first takes the oldest of them: the plan's stream waits for
 * its copies and the call computes on it.  So with stage(i + 1) issued before call(i), step
 * i + 1's data are copied while step i computes.  The plan holds a second set of eigen-data
 * buffers (allocated on the first staging); a staged set lands in whichever of the two sets no
 * later call reads, after the work already enqueued on the plan's stream.  From page-locked
 * host memory the copies run alongside the kernels; from pageable memory this call returns
 * only once the arrays have been read.  The host arrays must stay unchanged until the plan's
 * stream has passed the call that takes them (for a call with host outputs: until it has
 * returned).  chi0_plan_update drops the staged sets that no call has taken.  Errors:
 * CHI0_EINVAL (NULL plan or energies, evecs NULL without CMA, energies not ascending, a plan
 * with device inputs, two staged sets waiting already), CHI0_ENOMEM, CHI0_ECUDA. */
int chi0_plan_stage(chi0_plan_t *plan, const double *energies, const void *evecs);

/* Static chi0(q, w = 0) (Eq. 1 at w = 0, Sec. III) for nq q points: chi[iq].
 * Errors: CHI0_EINVAL (nq <= 0, NULL pointers, shift on a non-periodic grid, window
 * outside the plan's), CHI0_ECUDA, CHI0_ETIMEOUT (a tensor-core overlap wait ran out of
 * opts.wait_budget; the results of the call are then undefined, the plan stays usable). */
int chi0_static(chi0_plan_t *plan, const chi0_q_t *q, int nq, double *chi);

/* Static chi0 as chi0_static, and its band-pair contributions (the two-dimensional histogram
 * of Sec. III, Fig. 8: the part of chi0(q) from transitions m -> n):
 *   pairs[off_q + (m - lo_q) * w_q + (n - lo_q)],  w_q = hi_q - lo_q,
 * with the q blocks back to back (off_q = sum of w^2 over the q before it).  Occupied band m
 * at k, empty band n at k+q (Eq. 1), the normalisation and sign of chi; at a q flagged
 * Gamma the intraband pairs (m, m) carry the q -> 0 limit N(eF) of band m (Sec. III).  The
 * pairs of a q add up to chi[iq].  Each pair is summed in 64-bit fixed point (units of
 * 2^-50 before the normalisation: exact in any order, reproducible, one rounding of 2^-51
 * per term).  pairs is a host or device pointer like chi (opts.outputs_on_device) with room
 * for sum_q w_q^2 doubles; the call does not use graph capture.  Errors as chi0_static, plus
 * CHI0_EINVAL for pairs NULL or a plan window wider than 1024 bands.  The paper's figure is
 * a plot of these numbers; this entry point has no other counterpart in it. */
int chi0_static_pairs(chi0_plan_t *plan, const chi0_q_t *q, int nq, double *chi, double *pairs);

/* Dynamic chi0(q, w) (Eqs. 1-3) on nw frequencies: re[iq*nw + iw], im[iq*nw + iw].
 * Re is the principal value of Eq. 1; Im is Eq. 2 for w > 0, 0 at w = 0, and odd
 * (Eq. 3) for w < 0.  Errors as chi0_static, plus CHI0_EINVAL for nw <= 0. */
int chi0_dynamic(chi0_plan_t *plan, const chi0_q_t *q, int nq, const double *omega, int nw,
                 double *re, double *im);

/* Dynamic chi0 by the Kramers-Kronig route (Sec. II: Re obtained from Im, the usual way;
 * Eq. 1's principal value is what chi0_dynamic evaluates instead).  On the uniform grid
 * u_j = j wmax / (nkk - 1), j < nkk:
 *   im[iq*nkk + j]: Im chi0 (Eq. 2, the delta term alone: no logarithms, no principal value),
 *   re[iq*nkk + j]: (1/pi) PV int_0^wmax Im(u) [1/(u - u_j) + 1/(u + u_j)] du with Im taken
 *                   piecewise linear between the nodes and 0 from wmax on (exact for that
 *                   interpolant; at a Gamma q the intraband limit N(eF) is added at u = 0 as
 *                   chi0_dynamic adds it at w = 0).
 * The grid must cover the support of Im (wmax above the largest e_n(k+q) - e_m(k) of the
 * window): Sec. IV notes that the transform fails when it does not.  The error of Re against
 * the principal value falls with the grid spacing (second order where Im is smooth on the
 * grid's scale).  Im takes ceil(nkk / 256) passes of the weight kernel.  Errors as
 * chi0_dynamic, plus CHI0_EINVAL for wmax <= 0 or nkk < 2; the call does not use graph
 * capture.  re, im: host or device like chi0_dynamic's outputs. */
int chi0_dynamic_kk(chi0_plan_t *plan, const chi0_q_t *q, int nq, double wmax, int nkk, double *re, double *im);

/* Energies and eigenvectors at k+q for an off-grid q by linear interpolation from the plan's
 * mesh (Sec. II: the data at k+q are approximated by linear interpolation, energies and
 * matrix elements on equal footing).  For every corner k of the periodic mesh, k+q (qfrac in
 * units of the reciprocal lattice vectors) lies in one tetrahedron {000, e_p0, e_p0 + e_p1, 111}
 * of one cube (p: the axis order sorting the cube-local coordinates t descending); with the
 * barycentric weights (1 - t_p0, t_p0 - t_p1, t_p1 - t_p2, t_p2) every energy is the weighted
 * sum of the four corner values of its band, and every eigenvector the weighted sum of the four
 * corner vectors of its band after each is turned onto the phase of the first (times
 * conj(<v_0|v_i>) / |<v_0|v_i>|), normalised.  Outputs in the plan's layouts: e_kq [Nk][nbands]
 * (absolute energies, FP64), c_kq [Nk][norb][nbands] in the plan's eigenvector type (NULL, or
 * a CMA plan: energies only); device pointers when the plan takes device inputs, else host
 * pointers.  They are the explicit k+q data of a chi0_q_t (e_kq, c_kq) for chi0_static or
 * chi0_dynamic.  An approximation: its error falls with the mesh spacing (exact for data linear
 * in k).  Errors: CHI0_EINVAL (NULL plan, qfrac or e_kq, a non-periodic grid, |qfrac| >= 1e6),
 * CHI0_ENOMEM, CHI0_ECUDA. */
int chi0_interpolate_kq(chi0_plan_t *plan, const double *qfrac, double *e_kq, void *c_kq);

/* Autotuner.  Times the call (static when omega == NULL, else dynamic on nw frequencies)
 * once per candidate launch shape, with CUDA events on the plan's stream, and keeps the
 * fastest shape in the plan for its later calls.  Candidates, tuned one after the other:
 *   - block shape of the static weight kernel (threads and the register budget they
 *     leave) with its persistent CTAs per SM (1 .. the occupancy limit), or the persistent
 *     CTAs per SM of the dynamic weight kernel;
 *   - corners per MMA round of the tensor-core overlap (CHI0_OVL_BF16X3, BF16X6 or TF32 only;
 *     1, 2, 3, 4, 8, ... up to the most that fit one tile).
 * Every candidate computes the same chi0 up to rounding: the k-batch partials and their
 * summation order do not depend on the grid, and the corner grouping only changes how the
 * tensor-core FP32 accumulators are split.  Each timed call writes its results to chi / re,
 * im like chi0_static / chi0_dynamic.  *result: the chosen shape, the candidates timed, the
 * best and the untuned call times (ms).  Errors as chi0_static / chi0_dynamic. */
typedef struct {
  int static_variant;       /* block shape of the static weight kernel: FP32 0 = 256
                               threads x 2 blocks per SM (128 registers), 1 = 128 x 3,
                               2 = 256 x 1; FP64 always 0                           */
  int static_threads;       /* its threads per block                                */
  int static_ctas_per_sm;   /* persistent CTAs per SM of the static weight kernel  */
  int dynamic_ctas_per_sm;  /* ... of the dynamic weight kernel                     */
  int tc_corners_per_round; /* tensor-core overlap corner cap (0: most that fit)    */
  int candidates;           /* timed calls, the untuned one included                */
  double best_ms, default_ms;
} chi0_tune_t;
int chi0_tune(chi0_plan_t *plan, const chi0_q_t *q, int nq, const double *omega, int nw, double *re,
              double *im, chi0_tune_t *result);

/* Static chi0 without any device allocation (the paper has no counterpart: this is a
 * deployment variant of chi0_static).
 *
 * For callers that cannot call cudaMalloc where they need chi0: cudaMalloc/cudaFree can
 * synchronize the device and take unbounded time, which a real-time loop or a step with a
 * latency budget cannot afford, and some applications give all device memory to their own
 * pool allocator, which must account for every byte.  Such callers keep inputs and outputs
 * in memory they already own; this call uses a fixed work array inside the library instead.
 *
 *   kgrid  as for chi0_plan, but energies/evecs are DEVICE pointers; builtin tetrahedra.
 *   window band window [lo, hi) for m and n.
 *   opts   precision, cma, sign, tau, stream are used (inputs/outputs are always device).
 *   q[nq]  as for chi0_static; e_kq/c_kq, when given, are DEVICE pointers.
 *   chi    DEVICE pointer, [nq] results (same values as chi0_static on the same inputs).
 * Work memory: one array of CHI0_NOALLOC_SCRATCH_BYTES compiled into the library; every
 * GPU that loads the library holds it until the process exits.  A mesh whose work buffers
 * do not fit returns CHI0_EINVAL (chi0_last_error(NULL) states the bytes needed).  The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress, with that
 * device current); make that first call before any stream capture.  All calls share the
 * array and see the previous call's contents (what must start at zero is cleared on the
 * stream), so calls that overlap on the GPU race: serialize them on one stream.  The call
 * only enqueues work on opts->stream; it does not synchronize.  Errors: CHI0_EINVAL,
 * CHI0_ENOTSUP, CHI0_ECUDA; messages through chi0_last_error(NULL). */
#define CHI0_NOALLOC_SCRATCH_BYTES (64ull << 20)
int chi0_static_noalloc(const chi0_kgrid_t *kgrid, chi0_band_window_t window, const chi0_opts_t *opts,
                        const chi0_q_t *q, int nq, double *chi);

/* Measured arithmetic peak of the current device (a measurement helper for rooflines; the
 * paper has no counterpart).  kind: CHI0_PEAK_FP32_FMA / CHI0_PEAK_FP64_FMA (fused multiply-add
 * chains on the CUDA cores of every SM), CHI0_PEAK_TF32_MMA / CHI0_PEAK_BF16_MMA (back-to-back
 * tcgen05.mma, M = 128, N = 256, one 32-byte K step, from shared memory, one CTA per SM).
 * iters: loop length (the run should last some milliseconds: about 2e5 for the FMA kinds,
 * 2e5 for the MMA kinds).  One untimed warm-up launch, then one launch timed with CUDA events on
 * the legacy default stream; *tflops = 2 flop per FMA (or M N K per MMA) / time, *ms the time.
 * Synchronizes the device; allocates and frees a few bytes.  Errors: CHI0_EINVAL, CHI0_ENOMEM,
 * CHI0_ECUDA (including a bounded tensor-core wait that ran out). */
#define CHI0_PEAK_FP32_FMA 0
#define CHI0_PEAK_FP64_FMA 1
#define CHI0_PEAK_TF32_MMA 2
#define CHI0_PEAK_BF16_MMA 3
int chi0_peak(int kind, int iters, double *tflops, double *ms);

/* Copies the plan's accumulated counters into *stats.  CHI0_EINVAL on NULL. */
int chi0_plan_stats(const chi0_plan_t *plan, chi0_stats_t *stats);

/* Releases every device and host resource of the plan.  NULL-safe. */
void chi0_destroy(chi0_plan_t *plan);

/* Static-lifetime description of the last error of the plan (or of the last failed
 * chi0_plan call when plan == NULL). */
const char *chi0_last_error(const chi0_plan_t *plan);

/* Library ABI version (major*10000 + minor*100 + patch): 101 adds chi0_stats_t.queue_overflow
 * and chi0_stats_t.box_pieces; 102 adds chi0_static_pairs; 103 adds chi0_dynamic_kk; 104 adds chi0_interpolate_kq; 105 adds chi0_plan_update; 106 adds chi0_plan_stage. */
int chi0_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CHI0_H */
