// Internal declarations of the layer-potential operators (layer.cu) used by the evaluation engine.
#pragma once

#include <cuda_runtime.h>

namespace vp {

// One instance of a small dense operator on boundary point sources: the sources perm[j0 .. j0+ns)
// (each with two density components) map to `rows` outputs written at strided destinations. The
// matrix is stored column-major, [2 ns][rows], column 2 j + b for source j and component b.
//  coefficient builders: (cx, cy) circle centre, R sampling radius, r reference radius of the box;
//  near builder:         (cx, cy) lower-left corner of the target leaf, R its side.
struct PtInst {
  double cx, cy, R, r;
  int j0, ns;
  int kact;         // channel K of the far field active at the box's level
  int pad;
  long long aoff;   // matrix offset (elements)
  long long dst;    // destination base offset (elements)
};

// Boundary point sources: coordinates, unit normal (into the domain), quadrature weight, and the
// permutation that lists them leaf by leaf.
struct PtSources {
  const double *x, *y, *nx, *ny, *w;
  const int* perm;
};

// Multipole (kind 0) or local (kind 1) coefficients, both velocity components and both channels
// (rows a E + ch C + mode), of the double-layer field of each listed source, by sampling on a circle
// and a discrete Fourier transform. nch must be 2.
int launch_pt_coeffs(int kind, double alpha, int P, const PtInst* inst, int n_inst, int max_ns, PtSources src,
                     double* A, cudaStream_t s);
// Direct double-layer values at the p x p nodes of a target leaf (rows a n + node).
int launch_pt_near(double alpha, int p, const double* xi, const PtInst* inst, int n_inst, int max_ns,
                   PtSources src, double* A, cudaStream_t s);
// Y[dst + (row / rb) bs + row % rb] = sum over columns of A times the density (mu interleaved
// (mu_x, mu_y) per source), one block per instance; df != 0 writes double-float (two fp32) values,
// the slot format of split-precision trees, into the 8-byte elements of Y.
int launch_pt_apply(int rows, int rb, long long bs, int df, const PtInst* inst, int n_inst, const int* perm,
                    const double* mu, const double* A, double* Y, cudaStream_t s);

}  // namespace vp
