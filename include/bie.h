/*
 * bie.h -- C ABI of the boundary integral equation, its GMRES solver and the learned warm start
 * (libvp.so). Conventions as in vp.h: device pointers owned by the caller, `stream` a cudaStream_t,
 * return VP_OK (0) or a negative VP_ERR_* code.
 *
 * The homogeneous modified Stokes problem (af Klinteberg, Askham & Kropinski, Sec. 2.2) is
 * represented by the double-layer potential u^H = D[mu] (Eqs. uH_dbl, dbl_lyr_pot) with kernel
 * D_ij(x,y) = -T_jik(x-y) n_k(y) (Eq. dbl_lyr_ker), T the stresslet of App. B (Eq. app_stresslet),
 * n the unit normal pointing into the domain; the density solves the second-kind equation with the
 * nullspace correction W (Eq. BIE):  1/2 mu + D[mu] + W[mu] = g  on the boundary.
 * Boundary: the star r(t) = R + A cos(k t + phase), t in [0, 2 pi), counter-clockwise, split into
 * n_panels equal parameter panels of 16 Gauss-Legendre nodes (Sec. 3.2, Eq. BIE_quad); N =
 * 16 n_panels nodes, 2N unknowns ordered (mu_x, mu_y) per node.
 */
#ifndef BIE_H_
#define BIE_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bie_s* bie;

/*
 * bie_create -- nodes and the dense FP64 Nystrom matrix (2N x 2N, on the device) for alpha > 0.
 * Entries from the target's own panel and its two neighbours come from a graded local quadrature
 * of the kernel against the panel's Lagrange basis (the kernel's r log r terms); the rest are plain
 * Gauss-Legendre. max_krylov (1..1000) sizes the GMRES work space. Synchronises `stream`.
 * Errors: VP_ERR_ARG (alpha <= 0, A >= R, n_panels outside 4..4096), VP_ERR_OOM, VP_ERR_CUDA.
 */
int bie_create(double alpha, double R, double A, int k, double phase, int n_panels, int max_krylov, void* stream,
               bie* out);
void bie_free(bie b);

/* Number of nodes N and the boundary length. */
int bie_size(bie b, int* n_nodes, double* boundary_length);

/* Node data, device array [7][N]: x, y, n_x, n_y (inward unit normal), quadrature weight, curvature, t. */
int bie_nodes(bie b, double* out, void* stream);

/* out = (1/2 + D + W) mu (device arrays of 2N; mu 16-byte aligned, else VP_ERR_ARG). */
int bie_apply(bie b, const double* mu, double* out, void* stream);

/*
 * bie_solve -- GMRES (no restart; classical Gram-Schmidt applied twice, FP64) for (1/2+D+W) mu = g.
 *  g      device [2N] right-hand side.
 *  mu     device [2N], 16-byte aligned: initial guess on entry (zeros for a cold start), solution on return.
 *  tol    stop when the residual estimate <= tol * |g|;  max_iter <= max_krylov of bie_create.
 *  iters  receives the number of iterations; relres the true relative residual |g - A mu| / |g|.
 * The Arnoldi steps run on the device; the host queues four iterations at a time and reads the
 * device state between groups (steps queued past convergence do nothing). Synchronises `stream`.
 */
int bie_solve(bie b, const double* g, double* mu, double tol, int max_iter, int* iters, double* relres, void* stream);

/*
 * bie_solve_aug -- bie_solve with one augmentation direction d (device [2N], 16-byte aligned, or
 * NULL for plain bie_solve), e.g. a predicted correction to the initial guess. First the
 * least-squares step along d is taken (mu += s d with s minimising |r - s A d|); then GMRES runs on
 * the operator projected off c = A d / |A d| (each new Krylov vector loses its c component, whose
 * coefficients b_j are kept), and the final update is mu += V y - (b . y) d / |A d|. The residual
 * estimate of the projected Hessenberg system is the true residual, so the iteration stops at the
 * same tolerance, and the d direction stays resolved throughout. Same arguments and errors as
 * bie_solve otherwise.
 */
int bie_solve_aug(bie b, const double* g, double* mu, const double* d, double tol, int max_iter, int* iters,
                  double* relres, void* stream);

/* u = D[mu] at n_targets interior points txy [2][M] (plain quadrature: keep targets a few panel
 * lengths away from the boundary); u device [2][M]. */
int bie_eval(bie b, const double* mu, int n_targets, const double* txy, double* u, void* stream);

/* Sum of modified Stokes stokeslets (App. B, Eq. app_stokeslet): u(x) = sum_k S(x - src_k) f_k at
 * n_points xy [2][M]; src, f device [K][2]; u device [2][M]. Exact solutions for tests. */
int bie_stokeslets(double alpha, int n_sources, const double* src, const double* f, int n_points,
                   const double* xy, double* u, void* stream);

/* The scalar functions T1, T2, T3 (stresslet) and S1, S2 (stokeslet) of App. B at n arguments
 * z (device), out device [5][n] -- series of App. C for z <= 1.5, closed forms beyond. */
int bie_kernel_scalars(int n, const double* z, double* out, void* stream);

/*
 * Learned warm start (not in the paper): a circular 1D convolutional network over the boundary
 * nodes, FP32, layers of `width` channels and kernel `ksize` (odd), ReLU between layers:
 *   in_ch -> width -> ... -> width -> out_ch   (n_layers convolutions).
 * Parameters: for each layer l, weights [out][in][ksize] then bias [out], concatenated.
 * ws_create       initialises parameters (uniform, scaled by fan-in, seeded) and Adam state.
 * ws_num_params   number of parameters.
 * ws_params       copy parameters to (get != 0) or from (get == 0) a device float array.
 * ws_forward      y [B][out_ch][n] = net(x [B][in_ch][n]), device arrays.
 * ws_grad         forward + backward of the loss mean((y - t)^2) over all outputs; writes the
 *                 parameter gradient to grad (device, ws_num_params floats) and the loss (host).
 * ws_train_step   ws_grad followed by one Adam step (lr, beta1 0.9, beta2 0.999, eps 1e-8).
 * All asynchronous except that ws_grad / ws_train_step synchronise to return the loss.
 */
typedef struct ws_s* ws_net;
int ws_create(int in_ch, int width, int out_ch, int n_layers, int ksize, int n, int max_batch, uint64_t seed,
              void* stream, ws_net* out);
void ws_free(ws_net net);
int ws_num_params(ws_net net, int64_t* count);
int ws_params(ws_net net, float* buf, int get, void* stream);
int ws_forward(ws_net net, const float* x, int batch, float* y, void* stream);
int ws_grad(ws_net net, const float* x, const float* t, int batch, float* grad, float* loss, void* stream);
int ws_train_step(ws_net net, const float* x, const float* t, int batch, float lr, float* loss, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* BIE_H_ */
