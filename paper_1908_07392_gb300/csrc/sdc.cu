// Semi-implicit spectral deferred correction time stepping (Sec. 3.3; Eqs. sisdc_initial,
// sisdc_formula, rhs_initial, rhs_correction, rhs_correction_integral) of the Navier-Stokes equations
//   u_t + (u . grad) u = Laplacian u / Re - grad p,  div u = 0
// on a periodic box, every implicit substep solved by the periodic modified Stokes solution
// (vp_periodic: (alpha^2 - Laplacian) u + Re grad p = F, alpha^2 = Re / dt).
//
// Order K >= 2 takes p = K - 1 equal substeps dt = Delta t / p and K - 1 correction passes after the
// first pass of IMEX Euler substeps; order 1 is one IMEX Euler step of Delta t. Per node j of a pass
// the device keeps u_j, N_j = (u_j . grad) u_j and the implicit term L_j = Laplacian u_j - Re grad p_j,
// recovered after each solve as alpha^2 u_j - F_j. Node 0 of every pass is the state at the start of
// the step; at the first time L is the caller's Laplacian of u (a gradient in F does not change u).
// The quadrature of the correction right-hand side uses the integrals over [m, m + 1] of the Lagrange
// polynomials on the integer nodes 0..p, computed on the host in exact rational form.
//
// Every step runs on the caller's stream without host synchronisation: per substep one right-hand
// side kernel, the periodic solve, one kernel forming N and L from the solve's output.
#include <cuda_runtime.h>

#include <cmath>
#include <new>

#include "vp_internal.h"

#define TRY(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { set_last_cuda(e_); return e_ == cudaErrorMemoryAllocation ? VP_ERR_OOM : VP_ERR_CUDA; } } while (0)

namespace vp {
namespace {

constexpr int kMaxOrder = 4;
constexpr int kMaxNodes = kMaxOrder;  // p + 1 <= 4

// F = alpha^2 u_m - Re N_m (first pass, Eq. rhs_initial).
__global__ void k_sdc_rhs_first(long long n2, double alpha2, double re, const double* __restrict__ U,
                                const double* __restrict__ N, double* __restrict__ F) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x)
    F[i] = alpha2 * U[i] - re * N[i];
}

struct CorrArgs {
  long long n2;
  double alpha2, re;
  const double* u_new;   // u^{k+1}_m
  const double* n_new;   // N^{k+1}_m
  const double* n_old;   // N^k_m
  const double* l_next;  // L^k_{m+1}
  int nodes;             // p + 1
  double w[kMaxNodes];   // quadrature weights of the substep (q_j^m / dt)
  const double* lj[kMaxNodes];
  const double* nj[kMaxNodes];
  double* F;
};

// F = alpha^2 u^{k+1}_m - Re (N^{k+1}_m - N^k_m) - L^k_{m+1} + sum_j w_j (L^k_j - Re N^k_j)
// (correction pass, Eqs. rhs_correction, rhs_correction_integral).
__global__ void k_sdc_rhs_correct(CorrArgs a) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.n2;
       i += (long long)gridDim.x * blockDim.x) {
    double q = 0.0;
    for (int j = 0; j < a.nodes; ++j) q += a.w[j] * (a.lj[j][i] - a.re * a.nj[j][i]);
    a.F[i] = a.alpha2 * a.u_new[i] - a.re * (a.n_new[i] - a.n_old[i]) - a.l_next[i] + q;
  }
}

// After a solve: N = (u . grad) u from u [2][nn] and its gradient g [2][2][nn] (g[a][m] = du_a/dx_m),
// and (unless L is null) L = alpha^2 u - F.
__global__ void k_sdc_post(long long nn, double alpha2, const double* __restrict__ u, const double* __restrict__ g,
                           const double* __restrict__ F, double* __restrict__ N, double* __restrict__ L) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nn; i += (long long)gridDim.x * blockDim.x) {
    const double ux = u[i], uy = u[nn + i];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      N[c * nn + i] = ux * g[(2 * c) * nn + i] + uy * g[(2 * c + 1) * nn + i];
      if (L) L[c * nn + i] = alpha2 * u[c * nn + i] - F[c * nn + i];
    }
  }
}

// Integral over [m, m + 1] of the Lagrange polynomial of node j on the integer nodes 0..p: the
// polynomial's coefficients by expanding prod_{k != j} (s - k) / (j - k), then integrated term by
// term (all exact in FP64 for p <= 3: small integers over small denominators).
void quadrature_weights(int p, double w[kMaxOrder][kMaxNodes]) {
  for (int j = 0; j <= p; ++j) {
    double c[kMaxNodes + 1] = {1.0};  // c[d] = coefficient of s^d
    int deg = 0;
    double den = 1.0;
    for (int k = 0; k <= p; ++k) {
      if (k == j) continue;
      for (int d = deg + 1; d >= 1; --d) c[d] = c[d - 1] - k * c[d];
      c[0] = -k * c[0];
      ++deg;
      den *= (double)(j - k);
    }
    for (int m = 0; m < p; ++m) {
      double s = 0.0;
      for (int d = deg; d >= 0; --d) s += c[d] * (std::pow(m + 1.0, d + 1) - std::pow((double)m, d + 1)) / (d + 1);
      w[m][j] = s / den;
    }
  }
}

unsigned grid_for(long long n) {
  const long long g = (n + 255) / 256;
  return (unsigned)(g < 152 * 16 ? g : 152 * 16);
}

}  // namespace
}  // namespace vp

using namespace vp;

struct vp_sdc_s {
  double re = 0.0, dt_step = 0.0, alpha2 = 0.0;
  int order = 0, p = 0, n = 0;
  long long nn = 0;
  vp_periodic plan = nullptr;
  double* state[3] = {};                      // U, N, L at the start of the step
  double* node[2][kMaxNodes][3] = {};         // pass, node j >= 1, (U, N, L)
  double* F = nullptr;                        // [2][nn]
  double* G = nullptr;                        // [2][2][nn]: gradient of the latest solve
  double w[kMaxOrder][kMaxNodes] = {};
  bool has_state = false;                     // vp_sdc_set has been called
};

namespace {

int solve_node(vp_sdc_s* S, double* U, double* N, double* L, cudaStream_t s) {
  const int rc = vp_periodic_eval(S->plan, S->F, U, S->G, s);
  if (rc) return rc;
  k_sdc_post<<<grid_for(S->nn), 256, 0, s>>>(S->nn, S->alpha2, U, S->G, S->F, N, L);
  TRY(cudaGetLastError());
  return VP_OK;
}

// array of (U, N, L) of node j in pass k (node 0 is the state at the start of the step)
double* const* node_of(vp_sdc_s* S, int pass, int j) { return j == 0 ? S->state : S->node[pass][j]; }

int one_step(vp_sdc_s* S, cudaStream_t s) {
  const long long n2 = 2 * S->nn;
  const int p = S->p;
  // first pass
  for (int m = 0; m < p; ++m) {
    double* const* a = node_of(S, 0, m);
    k_sdc_rhs_first<<<grid_for(n2), 256, 0, s>>>(n2, S->alpha2, S->re, a[0], a[1], S->F);
    TRY(cudaGetLastError());
    double* const* b = node_of(S, 0, m + 1);
    const int rc = solve_node(S, b[0], b[1], b[2], s);
    if (rc) return rc;
  }
  // correction passes, alternating the pass buffers
  int old = 0;
  const int n_corr = S->order >= 2 ? S->order - 1 : 0;
  for (int k = 0; k < n_corr; ++k) {
    const int nw = 1 - old;
    for (int m = 0; m < p; ++m) {
      CorrArgs c{};
      c.n2 = n2; c.alpha2 = S->alpha2; c.re = S->re;
      double* const* vn = node_of(S, nw, m);
      double* const* vo = node_of(S, old, m);
      c.u_new = vn[0]; c.n_new = vn[1]; c.n_old = vo[1];
      c.l_next = node_of(S, old, m + 1)[2];
      c.nodes = p + 1;
      for (int j = 0; j <= p; ++j) {
        c.w[j] = S->w[m][j];
        c.lj[j] = node_of(S, old, j)[2];
        c.nj[j] = node_of(S, old, j)[1];
      }
      c.F = S->F;
      k_sdc_rhs_correct<<<grid_for(n2), 256, 0, s>>>(c);
      TRY(cudaGetLastError());
      double* const* b = node_of(S, nw, m + 1);
      const int rc = solve_node(S, b[0], b[1], b[2], s);
      if (rc) return rc;
    }
    old = nw;
  }
  // the last node of the last pass becomes the state; its old arrays take that node's place
  for (int f = 0; f < 3; ++f) {
    double* t = S->state[f];
    S->state[f] = S->node[old][p][f];
    S->node[old][p][f] = t;
  }
  return VP_OK;
}

}  // namespace

extern "C" int vp_sdc_create(double re, double dt, int order, int n, double side, void* stream, vp_sdc* out) {
  if (!out) return VP_ERR_ARG;
  *out = nullptr;
  if (!(re > 0.0) || !(dt > 0.0) || order < 1 || order > kMaxOrder) return VP_ERR_ARG;
  vp_sdc_s* S = new (std::nothrow) vp_sdc_s();
  if (!S) return VP_ERR_OOM;
  S->re = re; S->dt_step = dt; S->order = order; S->n = n;
  S->p = order >= 2 ? order - 1 : 1;
  const double sub = dt / S->p;
  S->alpha2 = re / sub;
  S->nn = (long long)n * n;
  int rc = vp_periodic_create(std::sqrt(S->alpha2), n, side, stream, &S->plan);
  if (rc) { delete S; return rc; }
  auto fail = [&](int code) { vp_sdc_free(S); return code; };
  const size_t bytes2 = (size_t)2 * S->nn * sizeof(double);
  for (int f = 0; f < 3; ++f)
    if (cudaMalloc(&S->state[f], bytes2) != cudaSuccess) { cudaGetLastError(); return fail(VP_ERR_OOM); }
  const int passes = order >= 2 ? 2 : 1;
  for (int k = 0; k < passes; ++k)
    for (int j = 1; j <= S->p; ++j)
      for (int f = 0; f < 3; ++f)
        if (cudaMalloc(&S->node[k][j][f], bytes2) != cudaSuccess) { cudaGetLastError(); return fail(VP_ERR_OOM); }
  if (cudaMalloc(&S->F, bytes2) != cudaSuccess || cudaMalloc(&S->G, 2 * bytes2) != cudaSuccess) {
    cudaGetLastError();
    return fail(VP_ERR_OOM);
  }
  quadrature_weights(S->p, S->w);
  *out = S;
  return VP_OK;
}

extern "C" int vp_sdc_set(vp_sdc S, const double* u0, const double* gradu0, const double* lap0, void* stream) {
  if (!S || !u0 || !gradu0 || !lap0) return VP_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t bytes2 = (size_t)2 * S->nn * sizeof(double);
  TRY(cudaMemcpyAsync(S->state[0], u0, bytes2, cudaMemcpyDeviceToDevice, s));
  TRY(cudaMemcpyAsync(S->state[2], lap0, bytes2, cudaMemcpyDeviceToDevice, s));
  TRY(cudaMemcpyAsync(S->G, gradu0, 2 * bytes2, cudaMemcpyDeviceToDevice, s));
  // N of the initial state
  k_sdc_post<<<grid_for(S->nn), 256, 0, s>>>(S->nn, S->alpha2, S->state[0], S->G, nullptr, S->state[1], nullptr);
  TRY(cudaGetLastError());
  S->has_state = true;
  return VP_OK;
}

extern "C" int vp_sdc_step(vp_sdc S, int n_steps, void* stream) {
  if (!S || n_steps < 0 || !S->has_state) return VP_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < n_steps; ++i) {
    const int rc = one_step(S, s);
    if (rc) return rc;
  }
  return VP_OK;
}

extern "C" int vp_sdc_get(vp_sdc S, double* u, double* gradu, void* stream) {
  if (!S || !u || !gradu || !S->has_state) return VP_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t bytes2 = (size_t)2 * S->nn * sizeof(double);
  TRY(cudaMemcpyAsync(u, S->state[0], bytes2, cudaMemcpyDeviceToDevice, s));
  TRY(cudaMemcpyAsync(gradu, S->G, 2 * bytes2, cudaMemcpyDeviceToDevice, s));
  return VP_OK;
}

extern "C" void vp_sdc_free(vp_sdc S) {
  if (!S) return;
  vp_periodic_free(S->plan);
  for (double* p : S->state) if (p) cudaFree(p);
  for (auto& pass : S->node)
    for (auto& nd : pass)
      for (double* p : nd) if (p) cudaFree(p);
  if (S->F) cudaFree(S->F);
  if (S->G) cudaFree(S->G);
  delete S;
}
