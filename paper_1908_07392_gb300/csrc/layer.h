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

namespace vp {

// Near-boundary correction of the layer potential for sources that are the panel nodes of the star
// r(t) = R + A cos(k t + phase) (equal parameter panels of kNearQ Gauss-Legendre nodes).
constexpr int kNearQ = 16;
struct StarGeom { double R, A, phase; int k, n_panels; };
// One (target node, panel) pair: target coordinates, the panel, and the parameter of the closest
// point of the panel to the target with the distance.
struct NearPair { double x, y, t0, d; int panel, pad; };
// dW[pair][j][a][b] (j < kNearQ) = graded-quadrature weight of node j of the panel for velocity
// component a and density component b, minus the plain Gauss-Legendre weight of that node.
int launch_near_weights(double alpha, StarGeom g, const NearPair* pairs, long long n_pairs, double* dW,
                        cudaStream_t s);
// u[a][node] += sum over the node's pairs of dW times the density of the pair's panel nodes; node k of the
// list is `node[k]`, its pairs ptr[k] .. ptr[k+1].
int launch_near_apply(long long n_nodes, const long long* node, const long long* ptr, const int* panel,
                      const double* dW, const double* mu, long long N, double* u, cudaStream_t s);

}  // namespace vp
