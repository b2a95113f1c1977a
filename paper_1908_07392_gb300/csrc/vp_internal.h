// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/vp.h"

namespace vp {

// Number of relative positions of each operator family.
constexpr int kNearPos = 33;  // U list: self, 8 same-level, 12 coarser, 12 finer adjacent leaves
constexpr int kWPos = 20;     // W list: level l+1 children of colleagues, not adjacent
constexpr int kXPos = 20;     // X list: level l-1 leaves adjacent to the parent, not to the box
constexpr int kVOff = 40;     // V list: same-level offsets in [-3,3]^2 \ [-1,1]^2
constexpr int kSpecialMaxOrder = 64;  // highest order vp_special evaluates

// Source box relative to a target box [0,1]^2 (units of the target side):
// lower-left (ox, oy) and side s.
struct RelBox {
  double ox, oy, s;
};

// Enumerations of the relative positions (built once, host side).
struct Positions {
  RelBox near[kNearPos];
  RelBox w[kWPos];
  RelBox x[kXPos];
  int v_dx[kVOff], v_dy[kVOff];
  // lookup tables from integer relative coordinates to indices (-1 = invalid)
  int near_same[3][3];   // [dy+1][dx+1]
  int near_coarse[4][4]; // [Y+2][X+2], X,Y in units of the target side
  int near_fine[4][4];   // [Y+1][X+1], X,Y in units of half the target side
  int w_idx[6][6];       // [Y+2][X+2], half units
  int x_idx[6][6];       // [Y+3][X+3], target units
  int v_idx[7][7];       // [dy+3][dx+3]
};
const Positions& positions();

// Expansion modes of one channel: index 0 -> m = 0, 1..P -> cos(m theta), P+1..2P -> sin(m theta).
// Channel 0 (K): multipole K_m(alpha rho)/K_m(alpha r_l), local I_m(alpha rho)/I_m(alpha r_l).
// Channel 1 (L, modified-biharmonic kernel only): multipole log rho, (r_l/rho)^m; local (rho/r_l)^m.
// r_l = h_l / sqrt(2) is the circumradius of a level-l box.

// Last CUDA error seen by the library (for diagnostics).
void set_last_cuda(cudaError_t e);
cudaError_t last_cuda();

// Gauss-Legendre nodes and weights on [-1, 1], ascending (host).
void gauss_legendre_host(int n, double* x, double* w);

}  // namespace vp


struct vp_tables_s {
  int kernel = 0;
  double alpha = 0.0;
  int p = 0, n = 0;      // nodes per side, nodes per leaf
  int P = 0, C = 0;      // expansion order, coefficients per channel (2P+1)
  int nch = 1, E = 0;    // channels, coefficients per box (nch*C)
  int levels = 0;        // deepest leaf level served
  int precision = VP_PREC_FP64;
  double side = 0.0;
  std::vector<int> kactive;  // per level: K-channel far field active
  // device tables (layouts in tables.cu)
  double* near = nullptr;    // [L+1][33][3n][n]
  double* s2m = nullptr;     // [L+1][E][n]
  double* l2t = nullptr;     // [L+1][3n][E]
  double* m2m = nullptr;     // [L+1][nch][C][4C]        (parent level)
  double* l2l = nullptr;     // [L+1][4][nch][C][C]      (parent level)
  double* m2l = nullptr;     // [L+1][40][nch][C][C]
  double* m2t = nullptr;     // [L+1][20][nch][3n][C]    (target level; source l+1)
  double* s2l = nullptr;     // [L+1][20][nch][C][n]     (target level; source leaf l-1)
  // VP_PREC_SPLIT: sliced copies of the operator tables (vp::SplitTables, split.cu)
  void* near_split = nullptr;
  int n_slices = 0;

  size_t near_stride_pos() const { return (size_t)3 * n * n; }
  size_t near_stride_lvl() const { return near_stride_pos() * vp::kNearPos; }
  size_t s2m_stride_lvl() const { return (size_t)E * n; }
  size_t l2t_stride_lvl() const { return (size_t)3 * n * E; }
  size_t m2m_stride_ch() const { return (size_t)C * 4 * C; }
  size_t m2m_stride_lvl() const { return m2m_stride_ch() * nch; }
  size_t l2l_stride_ch() const { return (size_t)C * C; }
  size_t l2l_stride_q() const { return l2l_stride_ch() * nch; }
  size_t l2l_stride_lvl() const { return l2l_stride_q() * 4; }
  size_t m2l_stride_ch() const { return (size_t)C * C; }
  size_t m2l_stride_off() const { return m2l_stride_ch() * nch; }
  size_t m2l_stride_lvl() const { return m2l_stride_off() * vp::kVOff; }
  size_t m2t_stride_ch() const { return (size_t)3 * n * C; }
  size_t m2t_stride_pos() const { return m2t_stride_ch() * nch; }
  size_t m2t_stride_lvl() const { return m2t_stride_pos() * vp::kWPos; }
  size_t s2l_stride_ch() const { return (size_t)C * n; }
  size_t s2l_stride_pos() const { return s2l_stride_ch() * nch; }
  size_t s2l_stride_lvl() const { return s2l_stride_pos() * vp::kXPos; }
  double h(int l) const { return side / (double)(1ll << l); }
};
