// chi0_overlap_tc.cu -- |M_mn(k,q)|^2 (the Eq. 1 matrix elements in the tight-binding form
// of the Sec. III footnote) on the 5th-generation tensor cores: tcgen05.mma with shared-memory
// operands and an FP32 accumulator in tensor memory.
//
// Per k corner c the overlap O = A^H B, A = C[c][:, lo:hi] (norb x w, complex), B the same
// block at k+q, is one real GEMM with K = 2 norb, real and imaginary parts interleaved along K
// (K index 2o: real part of orbital o, 2o + 1: imaginary part):
//   row m of the A operand:        (Re A[o][m], Im A[o][m])  for o = 0 .. norb-1
//   row n of the B operand (Re):   (Re B[o][n], Im B[o][n])          -> Re O[m][n]
//   row NW + n (Im):               (Im B[o][n], -Re B[o][n])         -> Im O[m][n]
// so that one accumulator row (one tensor-memory lane) holds both Re O[m][:] and Im O[m][:]
// and the epilogue forms |O|^2 without exchanging data between lanes.  Several corners share
// one MMA round: corner g's A rows sit at g*w .. g*w + w - 1 of the M = 128 tile and its B
// rows at g*2NW .. of the N <= 256 tile; the off-diagonal corner blocks of the product are
// computed and never read.
//
// Accumulation.  The tensor core adds each MMA's products to its FP32 accumulator with
// truncation, so every MMA accumulated into one place moves the result toward zero by a
// fraction of an ulp: measured on chi0, 6e-8 relative per MMA (3.2e-7 with 6 MMAs per
// element, 1.8e-6 with 30), a bias that the sum over k does not average away.  The K steps
// are therefore spread over NACC accumulators (tensor-memory column blocks of N: round-robin
// when all of K is staged at once, one contiguous chunk each otherwise), each accumulator
// takes its smallest products first and the leading piece product last, and the epilogue
// adds the NACC partial results on the CUDA cores (round to nearest).  With NACC equal to
// the number of K steps each accumulator sees one leading-order MMA.
//
// Precision forms (FP32 accumulation in all):
//   TF32    one product of round-to-nearest TF32 operands
//   BF16X3  x = p0 + p1 with p0 = bf16(x), p1 = bf16(x - p0); products p0 p0 + p0 p1 + p1 p0
//   BF16X6  x = p0 + p1 + p2 (p2 = bf16(x - p0 - p1)); the six products pa pb with a + b <= 2
//
// K chunks.  When the whole K extent of every piece does not fit in shared memory (the
// three-piece split at 80 orbitals: 3 (128 + 160) 320 bytes = 276 KB), K is cut into chunks of
// kc K steps, staged into two buffers in turn: the threads convert chunk j + 1 while the
// tensor core multiplies chunk j.  Each chunk goes to its own accumulator (chunks are
// contiguous runs of K steps), smallest products first, so that the truncation bias stays
// that of kc leading-order MMAs per accumulator.
//
// Operands are staged by the CTA's threads (conversion to TF32/BF16 and the real form above)
// into the K-major, non-swizzled tcgen05 layout: core matrices of 8 rows x 16 bytes stored as
// 128 contiguous bytes, core matrix (row group rb, 16-byte column kb) at (rb * KB + kb) * 128
// bytes (KB = 16-byte columns per row), so the descriptor strides are 128 bytes along K and
// KB * 128 bytes along M/N.  One thread issues the MMAs and commits them to an mbarrier; every
// wait on it is bounded (the plan's wait budget, in clock cycles) and a wait that runs out
// sets the error word, frees the tensor memory and ends the kernel.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "chi0_internal.h"

namespace chi0int {
namespace {

constexpr int kTcThreads = 256;  // 8 warps: warp i reads tensor-memory lanes 32(i%4) .. +31
constexpr int kTcM = 128;        // MMA rows (cta_group::1)
constexpr int kTcMaxN = 256;     // MMA columns
constexpr int kTcCols = 512;           // tensor-memory columns of an SM
constexpr int kTcMinSmem = 80 * 1024;  // at most 2 CTAs per SM when a CTA takes <= 256 columns
constexpr int kTcOneSmem = 116 * 1024; // one CTA per SM when it takes all 512 columns

struct TcShape {
  int w, NW, G, N, Kpad, Kbytes, ES, P, nks, NACC, ncols;
  int kc, nch, chunked;  // K steps per staged chunk, chunks per round, double-buffered chunks
  size_t smem;
};

// gcap > 0 caps the corners per round (the autotuner's candidates)
__host__ __device__ inline TcShape tc_shape(int w, int norb, int mode, int gcap) {
  TcShape s{};
  s.w = w;
  s.NW = (w + 7) & ~7;
  s.ES = mode == TC_TF32 ? 4 : 2;
  s.P = mode == TC_TF32 ? 1 : (mode == TC_BF16X3 ? 2 : 3);
  const int kstep = 32 / s.ES;  // K elements per MMA instruction (32 bytes of K)
  s.Kpad = (2 * norb + kstep - 1) / kstep * kstep;
  s.Kbytes = s.Kpad * s.ES;
  s.nks = s.Kbytes / 32;
  const int g1 = kTcM / (w > 0 ? w : 1), g2 = kTcMaxN / (2 * s.NW);
  s.G = g1 < g2 ? g1 : g2;
  if (s.G < 1) s.G = 0;  // window too wide for one tile
  if (gcap > 0 && s.G > gcap) s.G = gcap;
  if (mode != TC_TF32 && s.G > 1) {
    // fewer corners per round when that lets every K step have its own accumulator
    const int g3 = kTcCols / (2 * s.NW * s.nks);
    s.G = g3 < 1 ? 1 : (g3 < s.G ? g3 : s.G);
  }
  s.N = s.G * 2 * s.NW;
  s.NACC = mode == TC_TF32 ? 1 : (s.N > 0 ? kTcCols / s.N : 1);
  if (s.NACC > s.nks) s.NACC = s.nks;
  if (s.NACC < 1) s.NACC = 1;
  s.kc = s.nks;
  s.nch = 1;
  s.chunked = 0;
  s.smem = (size_t)s.P * (kTcM + s.N) * s.Kbytes + 64;
  if (s.G >= 1 && s.smem > kTcSmemMax) {
    // two chunk buffers; one accumulator per chunk where the tensor memory allows
    s.chunked = 1;
    s.kc = (s.nks + s.NACC - 1) / s.NACC;
    while (s.kc > 1 && 2 * (size_t)s.P * (kTcM + s.N) * s.kc * 32 + 64 > kTcSmemMax) --s.kc;
    s.nch = (s.nks + s.kc - 1) / s.kc;
    if (s.NACC > s.nch) s.NACC = s.nch;
    s.smem = 2 * (size_t)s.P * (kTcM + s.N) * s.kc * 32 + 64;
    if (s.smem > kTcSmemMax) s.G = 0;  // even one K step per chunk does not fit
  }
  int nc = 32;
  while (nc < s.NACC * s.N) nc <<= 1;
  s.ncols = nc;
  return s;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, leading (K) and stride (M/N) byte offsets,
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

// instruction descriptor: FP32 accumulator, TF32 or BF16 operands, both K-major, M = 128
__device__ __forceinline__ uint32_t idesc(int mode, int N) {
  const uint32_t ab = mode == TC_TF32 ? 2u : 1u;
  return (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc, int mode) {
  if (mode == TC_TF32)
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(id), "r"(acc));
  else
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(id), "r"(acc));
}

// 8 consecutive FP32 columns of this thread's tensor-memory lane (load and wait in one block)
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float v[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// byte offset of element (row r, column k) in a K-major core-matrix tile
__device__ __forceinline__ uint32_t tile_off(int r, int k, int ES, int KB) {
  const int kb = k * ES;
  return (uint32_t)(((r >> 3) * KB + (kb >> 4)) * 128 + (r & 7) * 16 + (kb & 15));
}

// store x at (r, k) of every piece of a tile (pieces are `stride` bytes apart)
template <int MODE>
__device__ __forceinline__ void put(unsigned char *base, size_t stride, int r, int k, int KB, float x) {
  if constexpr (MODE == TC_TF32) {
    *(uint32_t *)(base + tile_off(r, k, 4, KB)) = tf32_rn(x);
  } else {
    const uint32_t off = tile_off(r, k, 2, KB);
    constexpr int P = MODE == TC_BF16X3 ? 2 : 3;
    float rem = x;
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const __nv_bfloat16 h = __float2bfloat16_rn(rem);
      *(unsigned short *)(base + p * stride + off) = __bfloat16_as_ushort(h);
      rem -= __bfloat162float(h);
    }
  }
}

// Bounded wait on an mbarrier phase; false when the budget (clock cycles) ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long budget) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > budget) return false;
  }
}

// Stages orbitals [o0, o1) of the round's corners c0 .. c0 + G - 1 into one operand buffer
// (P pieces of A, then P pieces of B; KB 16-byte columns per row): element (g, o, band) goes
// to A row g*w + m and B rows g*2NW + n, g*2NW + NW + n at K columns 2(o - o0) and 2(o - o0) + 1.
// kUnroll elements per thread and pass: all their loads are issued before the first store.
template <int MODE, typename CTq>
__device__ __forceinline__ void stage_orbitals(const Grid &g, const float2 *__restrict__ C,
                                               const CTq *__restrict__ Cb, int explicit_q, const Q &q,
                                               const TcShape &sh, long long c0, int o0, int o1,
                                               unsigned char *sA, unsigned char *sB, size_t a_piece,
                                               size_t b_piece, int KB) {
  const int w = sh.w, NW = sh.NW, no = g.norb, nob = o1 - o0;
  const int per = nob * w, tot = sh.G * per;
  constexpr int kUnroll = 4;
  for (int i0 = threadIdx.x; i0 < tot; i0 += kUnroll * kTcThreads) {
    float2 xv[kUnroll];
    CTq yv[kUnroll];
    int ra[kUnroll], rb[kUnroll], kk[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int i = i0 + u * kTcThreads;
      const int gg = i / per, rem = i - gg * per;
      const long long c = c0 + gg;
      ra[u] = -1;
      if (i >= tot || c >= g.nc) continue;
      const int ol = rem / w, mm = rem - ol * w;
      const int o = o0 + ol;
      const long long ck = explicit_q ? c : shift_corner(g, c, q.shift);
      xv[u] = C[(c * no + o) * g.nb + q.lo + mm];
      yv[u] = Cb[(ck * no + o) * g.nb + q.lo + mm];
      ra[u] = gg * w + mm;
      rb[u] = gg * 2 * NW + mm;
      kk[u] = 2 * ol;
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      if (ra[u] < 0) continue;
      const float yr = (float)yv[u].x, yi = (float)yv[u].y;
      const int k = kk[u];
      put<MODE>(sA, a_piece, ra[u], k, KB, xv[u].x);
      put<MODE>(sA, a_piece, ra[u], k + 1, KB, xv[u].y);
      put<MODE>(sB, b_piece, rb[u], k, KB, yr);
      put<MODE>(sB, b_piece, rb[u], k + 1, KB, yi);
      put<MODE>(sB, b_piece, rb[u] + NW, k, KB, yi);
      put<MODE>(sB, b_piece, rb[u] + NW, k + 1, KB, -yr);
    }
  }
}

// Zeroes K columns [k0, k1) of the rows a round uses (a chunk buffer that held a longer chunk
// before: its K padding must read as zero).
template <int MODE>
__device__ __forceinline__ void zero_columns(const TcShape &sh, int k0, int k1, unsigned char *sA,
                                             unsigned char *sB, size_t a_piece, size_t b_piece, int KB) {
  const int na = sh.G * sh.w, nbr = sh.N, nk = k1 - k0;
  const int tot = (na + nbr) * nk;
  for (int i = threadIdx.x; i < tot; i += kTcThreads) {
    const int r = i / nk, k = k0 + (i - r * nk);
    if (r < na) put<MODE>(sA, a_piece, r, k, KB, 0.0f);
    else put<MODE>(sB, b_piece, r - na, k, KB, 0.0f);
  }
}

template <int MODE, typename CTq>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_overlap_tc(Grid g, const float2 *__restrict__ C, const CTq *__restrict__ Cb, int explicit_q, Q q,
                 float *__restrict__ W2, long long budget, int test_stall, int gcap, int *__restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const TcShape sh = tc_shape(q.hi - q.lo, g.norb, MODE, gcap);
  const int w = sh.w, NW = sh.NW, G = sh.G;
  // operand buffers: one holding all of K, or two holding one chunk of kc K steps each
  const int cbytes = sh.chunked ? sh.kc * 32 : sh.Kbytes;  // K bytes per row of a buffer
  const int KB = cbytes / 16;
  const size_t a_piece = (size_t)kTcM * cbytes, b_piece = (size_t)sh.N * cbytes;
  const size_t buf_bytes = sh.P * (a_piece + b_piece);
  const int nbuf = sh.chunked ? 2 : 1;
  unsigned char *tail = smem + nbuf * buf_bytes;
  uint64_t *bar = (uint64_t *)tail;
  uint32_t *tslot = (uint32_t *)(tail + 16);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int kOrbStep = MODE == TC_TF32 ? 4 : 8;  // orbitals per K step (32 bytes of K)
  const int ostep = kOrbStep * sh.kc;                 // orbitals per chunk

  // operand memory starts at zero: padding rows and K columns are never written again
  // (except a chunk buffer's K padding, cleared where a longer chunk used the buffer before)
  const size_t nz = (nbuf * buf_bytes) / 16;
  for (size_t i = tid; i < nz; i += blockDim.x) ((uint4 *)smem)[i] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(sh.ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t id = idesc(MODE, sh.N);
  const long long nround = (g.nc + G - 1) / G;
  uint32_t parity = 0;
  bool ok = true;
  // stages chunk j of the round starting at corner c0 into buffer j % nbuf
  auto stage = [&](long long c0, int j) {
    unsigned char *sA = smem + (j % nbuf) * buf_bytes;
    unsigned char *sB = sA + sh.P * a_piece;
    const int o0 = j * ostep, o1 = min(g.norb, o0 + ostep);
    stage_orbitals<MODE, CTq>(g, C, Cb, explicit_q, q, sh, c0, o0, o1, sA, sB, a_piece, b_piece, KB);
    // the last chunk of three or more may sit in a buffer whose K padding (inside its last K
    // step) an earlier, longer chunk filled
    if (sh.chunked && sh.nch >= 3 && j == sh.nch - 1) {
      const int kstep = 32 / sh.ES, kused = 2 * (o1 - o0);
      const int kpad = (kused + kstep - 1) / kstep * kstep;
      if (kused < kpad) zero_columns<MODE>(sh, kused, kpad, sA, sB, a_piece, b_piece, KB);
    }
    // generic-proxy stores must be visible to the tensor core's (async-proxy) reads
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  };
  // one thread issues chunk j's MMAs and commits them to the mbarrier
  auto issue = [&](int j) {
    if (tid != 0 || test_stall) return;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned char *sA = smem + (j % nbuf) * buf_bytes;
    const unsigned char *sB = sA + sh.P * a_piece;
    const int s0 = j * sh.kc, s1 = min(sh.nks, s0 + sh.kc);  // global K steps of the chunk
    for (int ia = 0; ia < sh.NACC; ++ia) {
      // unchunked: K step s goes to accumulator s % NACC; chunked: chunk j to j * NACC / nch
      if (sh.chunked && ia != j * sh.NACC / sh.nch) continue;
      // the first MMA into an accumulator in this round overwrites it
      uint32_t acc = (sh.chunked && j > 0 && (j - 1) * sh.NACC / sh.nch == ia) ? 1u : 0u;
      // products of pieces a, b with a + b = lvl < P, smallest level first
      for (int lvl = sh.P - 1; lvl >= 0; --lvl)
        for (int pa = 0; pa <= lvl; ++pa)
          for (int s = s0; s < s1; ++s) {
            if (!sh.chunked && s % sh.NACC != ia) continue;
            const uint32_t kb = (uint32_t)(s - s0) * 256u;  // 32 bytes of K = 2 core-matrix columns
            const uint64_t da = sdesc(smem_u32(sA + pa * a_piece) + kb, 128, KB * 128);
            const uint64_t db = sdesc(smem_u32(sB + (lvl - pa) * b_piece) + kb, 128, KB * 128);
            mma(tmem + (uint32_t)(ia * sh.N), da, db, id, acc, MODE);
            acc = 1;
          }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
  };
  for (long long rd = blockIdx.x; rd < nround && ok; rd += gridDim.x) {
    const long long c0 = rd * G;
    stage(c0, 0);
    __syncthreads();
    for (int j = 0; j < sh.nch; ++j) {
      issue(j);
      if (j + 1 < sh.nch) stage(c0, j + 1);  // the other buffer: chunk j - 1's MMAs are done
      // test_stall: nothing arrives, so the bounded wait below runs out (error path test).  The
      // CTA agrees on the outcome before any warp-wide tensor-memory load or buffer reuse.
      const int got = mbar_wait(smem_u32(bar), parity, budget) ? 1 : 0;
      if (!__syncthreads_and(got)) {
        ok = false;
        if (tid == 0) atomicExch(err, 1);
        break;
      }
      parity ^= 1u;
    }
    if (!ok) break;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // epilogue: lane r = gg*w + m of the tile holds Re O (columns gg*2NW + n) and Im O (+ NW);
    // warps i and i + 4 share lane quarter i%4 and split the 8-column chunks between them
    const int quarter = warp & 3, half = warp >> 2;
    const int r = quarter * 32 + lane;
    const int gg = r / (w > 0 ? w : 1), m = r - gg * w;
    const long long c = c0 + gg;
    const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16);
    for (int blk = 0; blk < G; ++blk) {  // warp-uniform loops: every lane takes part in tcgen05.ld
      for (int n0 = half * 8; n0 < NW; n0 += 16) {
        float re[8], im[8];
        tmem_ld8(trow + blk * 2 * NW + n0, re);
        tmem_ld8(trow + blk * 2 * NW + NW + n0, im);
        for (int ia = 1; ia < sh.NACC; ++ia) {  // partial accumulators, added in FP32
          float r2[8], i2[8];
          tmem_ld8(trow + ia * sh.N + blk * 2 * NW + n0, r2);
          tmem_ld8(trow + ia * sh.N + blk * 2 * NW + NW + n0, i2);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            re[j] += r2[j];
            im[j] += i2[j];
          }
        }
        if (blk == gg && gg < G && c < g.nc) {
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (n0 + j < w) W2[(c * w + m) * w + n0 + j] = re[j] * re[j] + im[j] * im[j];
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  if (!ok) {
    // the MMAs this CTA issued (if any) may still be running: wait for them once more,
    // bounded, before the tensor memory is released.  (The error-path test issues no MMA, so
    // there the second wait runs out as well and nothing is in flight.)
    mbar_wait(smem_u32(bar), parity, budget);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(sh.ncols) : "memory");
}

template <int MODE, typename CTq>
cudaError_t launch_tc(const Grid &g, const float2 *Ck, const CTq *Cb, int explicit_q, const Q &q, float *W2,
                      long long budget, int test_stall, int gcap, int *err, cudaStream_t s) {
  const TcShape sh = tc_shape(q.hi - q.lo, g.norb, MODE, gcap);
  const size_t floor_smem = sh.ncols > 256 ? (size_t)kTcOneSmem : (size_t)kTcMinSmem;
  const size_t smem = sh.smem < floor_smem ? floor_smem : sh.smem;
  cudaError_t e = cudaFuncSetAttribute(k_overlap_tc<MODE, CTq>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long nround = (g.nc + sh.G - 1) / sh.G;
  const int per_sm = smem > (size_t)113 * 1024 ? 1 : 2;
  long long blocks = (long long)sms * per_sm;
  if (blocks > nround) blocks = nround;
  k_overlap_tc<MODE, CTq><<<(int)blocks, kTcThreads, smem, s>>>(g, Ck, Cb, explicit_q, q, W2, budget, test_stall,
                                                                gcap, err);
  return cudaGetLastError();
}

// Tensor-core throughput: one CTA per SM issues `iters` MMAs (M = 128, N = 256, one K step of
// 32 bytes) from fixed zeroed shared-memory operands into one tensor-memory accumulator, then
// commits them and waits (bounded).  The large shared-memory request keeps one CTA per SM.
constexpr int kPeakSmem = 160 * 1024;
__global__ void __launch_bounds__(128, 1) k_tc_peak(int mode, int iters, long long budget, int *err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  constexpr int kN = 256;
  unsigned char *sA = smem, *sB = smem + kTcM * 32;
  uint64_t *bar = (uint64_t *)(sB + kN * 32);
  uint32_t *tslot = (uint32_t *)(sB + kN * 32 + 16);
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int i = tid; i < (kTcM + kN) * 32 / 16; i += blockDim.x) ((uint4 *)smem)[i] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  if (tid == 0) {
    const uint64_t da = sdesc(smem_u32(sA), 128, 2 * 128), db = sdesc(smem_u32(sB), 128, 2 * 128);
    const uint32_t id = idesc(mode, kN);
    for (int i = 0; i < iters; ++i) mma(tmem, da, db, id, i > 0 ? 1u : 0u, mode);
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
  }
  const int got = mbar_wait(smem_u32(bar), 0, budget) ? 1 : 0;
  if (!__syncthreads_and(got)) {
    if (tid == 0) atomicExch(err, 1);
    mbar_wait(smem_u32(bar), 0, budget);  // the MMAs may still run: wait once more, bounded
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kN) : "memory");
}

}  // namespace

cudaError_t tc_peak(int mode, int iters, double *tflops, double *ms_out) {
  int *err = nullptr;
  cudaError_t e = cudaMalloc(&err, sizeof(int));
  if (e != cudaSuccess) return e;
  cudaMemset(err, 0, sizeof(int));
  e = cudaFuncSetAttribute(k_tc_peak, cudaFuncAttributeMaxDynamicSharedMemorySize, kPeakSmem);
  if (e != cudaSuccess) {
    cudaFree(err);
    return e;
  }
  const int sms = device_sms();
  const long long budget = 1LL << 32;  // about two seconds: far above the run's length
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_tc_peak<<<sms, 128, kPeakSmem>>>(mode, iters / 8 + 1, budget, err);  // warm-up
  cudaEventRecord(e0);
  k_tc_peak<<<sms, 128, kPeakSmem>>>(mode, iters, budget, err);
  cudaEventRecord(e1);
  e = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(err);
  if (e != cudaSuccess) return e;
  if (herr) return cudaErrorTimeout;
  const double kel = mode == TC_TF32 ? 8.0 : 16.0;  // K elements of one 32-byte K step
  const double flops = 2.0 * kTcM * 256.0 * kel * (double)iters * sms;
  *tflops = flops / (ms * 1e-3) / 1e12;
  *ms_out = ms;
  return cudaSuccess;
}

size_t overlap_tc_smem(int w, int norb, int mode) {
  const TcShape sh = tc_shape(w, norb, mode, 0);
  if (sh.G < 1) return (size_t)-1;
  return sh.smem;
}

int overlap_tc_max_corners(int w, int norb, int mode) { return tc_shape(w, norb, mode, 0).G; }

cudaError_t launch_overlap_tc(const Grid &g, const void *C32, int dtype, const Q &q, float *W2, int mode,
                              long long budget, int test_stall, int gcap, int *err, cudaStream_t s) {
  const int w = q.hi - q.lo;
  if (w < 1 || overlap_tc_smem(w, g.norb, mode) > kTcSmemMax || !err) return cudaErrorInvalidValue;
  const float2 *Ck = (const float2 *)C32;
  if (budget <= 0) budget = 1LL << 31;
  if (mode == TC_BF16X6) {
    if (q.Cq && dtype == DT_C128)
      return launch_tc<TC_BF16X6, double2>(g, Ck, (const double2 *)q.Cq, 1, q, W2, budget, test_stall, gcap, err, s);
    if (q.Cq)
      return launch_tc<TC_BF16X6, float2>(g, Ck, (const float2 *)q.Cq, 1, q, W2, budget, test_stall, gcap, err, s);
    return launch_tc<TC_BF16X6, float2>(g, Ck, Ck, 0, q, W2, budget, test_stall, gcap, err, s);
  }
  if (mode == TC_TF32) {
    if (q.Cq && dtype == DT_C128)
      return launch_tc<TC_TF32, double2>(g, Ck, (const double2 *)q.Cq, 1, q, W2, budget, test_stall, gcap, err, s);
    if (q.Cq) return launch_tc<TC_TF32, float2>(g, Ck, (const float2 *)q.Cq, 1, q, W2, budget, test_stall, gcap, err, s);
    return launch_tc<TC_TF32, float2>(g, Ck, Ck, 0, q, W2, budget, test_stall, gcap, err, s);
  }
  if (q.Cq && dtype == DT_C128)
    return launch_tc<TC_BF16X3, double2>(g, Ck, (const double2 *)q.Cq, 1, q, W2, budget, test_stall, gcap, err, s);
  if (q.Cq) return launch_tc<TC_BF16X3, float2>(g, Ck, (const float2 *)q.Cq, 1, q, W2, budget, test_stall, gcap, err, s);
  return launch_tc<TC_BF16X3, float2>(g, Ck, Ck, 0, q, W2, budget, test_stall, gcap, err, s);
}

}  // namespace chi0int
