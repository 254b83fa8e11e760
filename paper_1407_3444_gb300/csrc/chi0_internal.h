// chi0_internal.h -- interface between the C-ABI layer and the kernel translation unit.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace chi0int {

struct Grid {
  int n[3];   // cubes per axis
  int N[3];   // corners per axis
  int periodic;
  int nb, norb;
  long long nc;    // corners
  long long ntet;  // tetrahedra
  double ef;
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
                           void *W2, int fp64, cudaStream_t s);

// band bounds per corner: occ[c] (1 + highest occupied band), emp[c] (lowest empty band);
// E32 (optional) receives (float)(E - ef)
cudaError_t launch_bands(const double *E, long long nc, int nb, double ef, short *occ, short *emp, float *E32,
                         cudaStream_t s);

// static weights: one FP64 partial per batch of 32 tetrahedra into partial[static_batches];
// Ek/Ekq are the absolute FP64 energies (fp64) or the FP32 energies relative to eF (mixed);
// occ from the k energies, empq from the k+q energies; next: a device int (batch counter)
cudaError_t launch_static(const Grid &g, const Tet &tet, const void *Ek, const void *Ekq, const Q &q,
                          const void *W2, int cma, int fp64, float tau, const short *occ, const short *empq,
                          double *partial, int *next, int nblocks, unsigned long long *counters,
                          cudaStream_t s);
int static_persistent_blocks(int fp64);
long long static_batches(long long ntet);

// dynamic weights: partialR/partialI [nblocks][nw]
cudaError_t launch_dynamic(const Grid &g, const Tet &tet, const double *E, const Q &q, const void *W2,
                           int cma, int fp64, float tau, const double *omega, int nw, double *partialR,
                           double *partialI, int nblocks, unsigned long long *counters, cudaStream_t s);

// Gamma: intraband q -> 0 limit, tetrahedron DOS at eF: partial[nblocks]
cudaError_t launch_dos(const Grid &g, const Tet &tet, const double *E, int lo, int hi, double *partial,
                       int nblocks, cudaStream_t s);

// out[idx*stride_out + k] = scale * sum_b partial[b*nw + k] (+ scale * sum dos where omega == 0)
cudaError_t launch_reduce(const double *partial, int nblocks, int nw, double scale, const double *dos,
                          int ndos, const double *omega, double *out, cudaStream_t s);

int static_blocks();
int dynamic_blocks(int nw);
int dynamic_max_nw();

}  // namespace chi0int
