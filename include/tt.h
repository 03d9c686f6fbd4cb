/*
 * tt.h -- C ABI of libtt, the GB300 (sm_103a) gradient-residual engine for
 * SAXS/WAXS tensor tomography with a real even-order spherical-harmonic basis
 * (Mumott, arXiv 2504.16446).
 *
 * Model (Section "Methodology"):
 *   I_sjkc = sum_xyz P_sjk,xyz sum_i B_sci c_xyzi           Eq. (forward_model)
 *   B_sci  = segment mean of Y_i(R_s^T q(phi))               Eq. (projection_matrix)
 *   r      = A c - I                                         Eq. (residual)
 *   L      = sum W r^2,  grad L = 2 A^T (W r)                Eq. (opt_prob_general_form), a = 2
 * P is Joseph's method (Section "Projectors and basis sets"): rays march the
 * planes of the main axis of their direction, bilinear interpolation of the
 * four voxel centres around the ray on each plane, zero outside the volume,
 * step length a/|p_s,m| per plane.  The adjoint is the exact transpose of that
 * discretisation.
 *
 * Conventions shared by every entry point
 *   - Geometry follows Eq. (real_space_geom) with centred indices: voxel
 *     (x,y,z) sits at a*(x-(nx-1)/2, y-(ny-1)/2, z-(nz-1)/2) in the sample
 *     frame; ray (j,k) passes through b*(j-(nj-1)/2-dj) j_s + b*(k-(nk-1)/2-dk) k_s
 *     with direction p_s, where v_s = R_s^T v and R_s = R_beta(beta_s) R_alpha(alpha_s)
 *     (right-handed rotations about the outer and inner axes).
 *   - Real SH: orthonormal, even l only, no Condon-Shortley phase, polar axis +z,
 *     azimuth from +x towards +y; index i runs over l = 0,2,..,ell_max and
 *     m = -l..l.  K = (ell_max+1)(ell_max+2)/2.
 *   - Layouts (row-major, caller-owned DEVICE memory unless stated):
 *       volume   c[nx][ny][nz][K]      (channel innermost)
 *       data     I[n_proj][nj][nk][n_seg], weights W with the same layout
 *       basis    B[n_proj][n_seg][K]   (FP64)
 *     Every device pointer must be 16-byte aligned (any cudaMalloc / torch
 *     allocation is).  Internal padding of K is invisible to the caller.
 *   - Element type: float for a TT_F32, TT_BF16 or TT_F16 handle, double for a
 *     TT_F64 handle (entry points with the _f64 suffix).  Calling the other
 *     kind returns TT_INVALID_ARG.
 *   - All work is enqueued on the handle's stream, in stream order.  Only
 *     entry points that return a host value (loss) synchronise that stream.
 *   - Inputs are never modified, except arguments named *_inout.
 *   - Errors are returned as tt_status; nothing aborts or throws across the
 *     ABI.  tt_last_error() gives a message for the calling thread.
 *   - Handles are not thread-safe; use one handle per host thread.
 */
#ifndef TT_H
#define TT_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TT_OK = 0,
    TT_INVALID_ARG = 1,       /* bad size, pointer, alignment, geometry or precision */
    TT_UNSUPPORTED = 2,       /* e.g. ell_max outside the compiled set */
    TT_OUT_OF_MEMORY = 3,     /* device or pinned-host allocation failed */
    TT_NONFINITE = 4,         /* the loss (hence some input) is NaN or infinite */
    TT_LINESEARCH_FAILED = 5, /* no Armijo point within the evaluation limit */
    TT_CUDA_ERROR = 6         /* a CUDA runtime call or kernel launch failed */
} tt_status;

/* Precision of a handle.  TT_F32 and TT_F64: storage and arithmetic in that
 * type.  TT_BF16 and TT_F16 (the reduced-precision form): the entry points
 * take and return float like TT_F32, but the coefficient volume that the
 * forward projector marches through is stored inside the path as bfloat16 /
 * float16 (halving the projector's volume traffic and footprint), with float
 * arithmetic and FP64 loss and dot-product reductions; the back-contracted
 * residual stays float.  Their results differ from FP32 by the 2-byte
 * rounding of the volume (relative ~1e-3 for bfloat16, ~1e-4 for float16). */
typedef enum { TT_F32 = 0, TT_F64 = 1, TT_BF16 = 2, TT_F16 = 3 } tt_precision;

/* Unit vectors of the instrument in laboratory coordinates, Table
 * "geometry_vectors": beam p, raster directions j and k, detector azimuth
 * origin q0 and +90 deg direction q90, inner (rotation) axis alpha and outer
 * (tilt) axis beta.  p, j, k must be orthonormal, and so must q0, q90 (both
 * orthogonal to p); the axes must be non-zero (they are normalised). */
typedef struct {
    double p[3], j[3], k[3], q0[3], q90[3], inner_axis[3], outer_axis[3];
} tt_frame;

/* Problem description, after the paper's data format (Table "h5_format").
 * All pointers are HOST arrays, copied by tt_create. */
typedef struct {
    int nx, ny, nz;              /* volume shape (voxels), each >= 1            */
    int nj, nk;                  /* raster pixels per projection, each >= 1    */
    int n_proj;                  /* projections s, 1..65535                     */
    int ell_max;                 /* even band limit, 0..12                      */
    int n_seg;                   /* detector segments c, 1..64                  */
    const double *inner_angle;   /* alpha_s [n_proj], radians                   */
    const double *outer_angle;   /* beta_s  [n_proj], radians                   */
    const double *j_offset;      /* delta j [n_proj], pixels; NULL = zeros      */
    const double *k_offset;      /* delta k [n_proj], pixels; NULL = zeros      */
    const double *seg_start;     /* phi_c,start [n_seg], radians                */
    const double *seg_end;       /* phi_c,end   [n_seg], radians, > start       */
    double two_theta;            /* scattering angle 2 theta, radians           */
    double voxel_size;           /* a > 0                                       */
    double step_size;            /* b >= a / 50                                 */
    tt_frame frame;
} tt_problem;

typedef struct tt_handle tt_handle;
typedef struct tt_lbfgs tt_lbfgs;
typedef struct tt_mitra tt_mitra;

/* Number of even-order real SH coefficients K for a band limit. */
int tt_num_coeffs(int ell_max);
const char *tt_status_string(tt_status s);
/* Message of the last failing call on this host thread ("" if none). */
const char *tt_last_error(void);

/* Limits checked here (TT_INVALID_ARG otherwise): nx*ny*nz <= 2^24 voxels,
 * 1 <= n_proj <= 65535, ell_max even and >= 0 (above 12: TT_UNSUPPORTED),
 * 1 <= n_seg <= 64, finite
 * angles and offsets, seg_end > seg_start, a > 0, b >= a / 50 (finer
 * detector pixels would put hundreds of rays on each voxel), orthonormal
 * p, j, k and q0, q90 _|_ p.
 * Validates the problem, copies it, computes the per-projection ray
 * constants (host, FP64) and the basis matrix (device, FP64, see
 * tt_basis_matrix), and allocates the handle's device scratch.  stream is a
 * cudaStream_t (NULL = legacy default stream); the current CUDA device at
 * this call is the handle's device.  The handle owns all of its memory. */
tt_status tt_create(const tt_problem *prob, tt_precision prec, void *stream, tt_handle **out);
tt_status tt_destroy(tt_handle *h);
/* Makes stream (cudaStream_t, NULL = legacy default stream) the handle's
 * stream for the calls that follow.  When it differs from the current one,
 * the new stream is ordered behind everything already enqueued on the old
 * stream (an event, no host synchronisation), so work still in flight there
 * (e.g. the adjoint behind an early-returned loss) is done with the handle's
 * buffers before the new stream reuses them. */
tt_status tt_set_stream(tt_handle *h, void *stream);
/* Chooses the kernel of the forward projection (Eq. forward_model, the
 * Joseph discretisation of Sec. "real_space_geom") for the calls that follow:
 *   0  automatic (the default): the tap-pair march (1), the faster of the
 *      two on every workload measured;
 *   1  the tap-pair march: bilinear taps read from the L1/L2-resident volume;
 *   2  the staged march: for each plane a copy warp moves the box of a ray
 *      tile's taps into shared memory with one tensor copy, and the rays read
 *      them there.  Applies to TT_F32 handles with 16 padded channels
 *      (ell_max 4) whose boxes fit the shared-memory ring (at most 32 voxels
 *      wide); TT_UNSUPPORTED otherwise.
 * Both compute the same FP32 ray sums (the same products added in the same
 * order), so projections and residual contractions agree bit for bit; the
 * loss is summed over ray tiles of different shapes and may differ in the
 * last bits.  Call it between evaluations on the handle's stream (it changes
 * only host state).  Other values: TT_INVALID_ARG. */
tt_status tt_set_forward_kernel(tt_handle *h, int kind);
/* Shape query: any out-pointer may be NULL. */
tt_status tt_get_sizes(const tt_handle *h, int *K, int *K_padded, long long *n_vox, long long *n_data);

/* Eq. (projection_matrix): B[s][c][i] = (1/dphi_c) * integral over segment c
 * of Y_i(R_s^T q(phi)) dphi, q(phi) = cos(theta)(cos phi q0 + sin phi q90) -
 * sin(theta) p, theta = two_theta/2, by a 32-node Gauss-Legendre rule per
 * segment, FP64, on the GPU.  Copies the handle's cached matrix into B_dev
 * (device, [n_proj][n_seg][K] doubles). */
tt_status tt_basis_matrix(tt_handle *h, double *B_dev);

/* The basis matrix of tt_basis_matrix without a handle and without allocating
 * device memory.  The paper has no counterpart: this entry point exists for
 * callers that cannot call cudaMalloc -- e.g. a process whose device memory is
 * owned and pre-reserved by another allocator, or code that must not trigger
 * the implicit device synchronisation of cudaMalloc/cudaFree.  Its scratch
 * (quadrature rule, rotated frames, segment bounds) is a fixed file-scope
 * device array of 18,624 doubles (145.5 KiB), present on every device that
 * loads libtt until the process exits; hence n_proj <= 2048 (n_seg <= 64,
 * ell_max <= 12 as for tt_create); larger problems return TT_INVALID_ARG.
 * prob is validated like tt_create's; B_dev (device, [n_proj][n_seg][K]
 * doubles, 16-byte aligned) receives the result, enqueued on stream
 * (cudaStream_t, NULL = legacy default stream).  The inputs are staged
 * through a per-thread pageable host buffer: the staging copy waits for the
 * work already enqueued on stream before it starts, and its bytes are staged
 * by the time the call returns.  The first call on each device looks up the
 * scratch array's device address (the device must be current); make that
 * first call before any stream capture.  All calls share the one scratch
 * array, which keeps the last call's contents; every call overwrites what it
 * reads, so nothing needs clearing, but calls whose work overlaps on the GPU
 * (other streams, other host threads) race on it. */
tt_status tt_basis_matrix_noalloc(const tt_problem *prob, double *B_dev, void *stream);

/* Forward model, Eq. (forward_model): I = A c.
 * c_dev [nx][ny][nz][K] -> I_dev [n_proj][nj][nk][n_seg]. */
tt_status tt_project(tt_handle *h, const float *c_dev, float *I_dev);
tt_status tt_project_f64(tt_handle *h, const double *c_dev, double *I_dev);

/* Adjoint of the forward model: g = A^T R (SH back-contraction with B_s,
 * then the exact transpose of the Joseph projection, a gather per voxel with
 * no atomics).  R_dev [n_proj][nj][nk][n_seg] -> g_dev [nx][ny][nz][K]. */
tt_status tt_adjoint(tt_handle *h, const float *R_dev, float *g_dev);
tt_status tt_adjoint_f64(tt_handle *h, const double *R_dev, double *g_dev);

/* Gradient-residual evaluation (Eq. residual with the squared loss):
 *   r = A c - I,  *loss_host = sum W r^2 (FP64 accumulation),
 *   g_dev = 2 A^T (W r).
 * W_dev may be NULL (all weights 1).  g_dev may be NULL (loss only).
 * c_dev may be NULL for c = 0: then *loss_host = sum W I^2 and g_dev =
 * -2 A^T (W I), the back-projection of the data, with the same results as
 * an all-zero c_dev, bit for bit, but without the forward projection (its
 * march over a zero volume is skipped; the contraction, residual and
 * back-contraction run as usual) -- the first evaluation of every solve
 * from zero and the learned warm start's input.
 * loss_host is a HOST pointer.  The call returns as soon as the loss is
 * known: with g_dev the adjoint publishes it in a page-locked slot when it
 * starts and may still be running on the handle's stream when the call
 * returns (g_dev is stream-ordered like every device output; c, I and W have
 * been consumed by then); without g_dev, or if no mapped slot could be
 * allocated, the call synchronises the stream.  Returns TT_NONFINITE (the
 * loss written, g following on the stream) when the loss is not finite. */
tt_status tt_gradient_residual(tt_handle *h, const float *c_dev, const float *I_dev,
                               const float *W_dev, float *g_dev, double *loss_host);
tt_status tt_gradient_residual_f64(tt_handle *h, const double *c_dev, const double *I_dev,
                                   const double *W_dev, double *g_dev, double *loss_host);

/* The same evaluation on HOST buffers (pageable or page-locked; W_host may
 * be NULL).  The inputs are staged through handle-owned device buffers: c
 * first, then I and W in up to eight projection chunks copied on a second
 * stream while the forward projects the chunks already present.  A
 * page-locked, device-mapped g_host (cudaHostAlloc / cudaMallocHost memory)
 * is written by the adjoint kernel in place; any other g_host receives the
 * gradient with one copy.  Same results, bit for bit, as
 * tt_gradient_residual.  Synchronous. */
tt_status tt_gradient_residual_host(tt_handle *h, const float *c_host, const float *I_host,
                                    const float *W_host, float *g_host, double *loss_host);

/* Regularisers (Section "Optimization": L2Norm, TotalVariation) of a volume
 * c_dev [nx][ny][nz][K] of the handle's shape; FP64 accumulation of the
 * value; grad_dev (may be NULL) receives the gradient; value_host is a HOST
 * pointer and the call synchronises the handle's stream.
 *   tt_l2_norm:  value = sum c^2, grad = 2 c.
 *   tt_tv_huber: value = sum over voxels x and channels i of H(|g_i(x)|),
 *     g_i(x)_d = c_i(x + e_d) - c_i(x) for x_d + 1 < N_d else 0 (forward
 *     differences, Neumann boundary), |.| Euclidean over d = x, y, z, and
 *     H(t) = t^2 / (2 delta) for t <= delta, t - delta/2 otherwise (delta > 0).
 * Returns TT_NONFINITE when the value is not finite. */
tt_status tt_l2_norm(tt_handle *h, const float *c_dev, float *grad_dev, double *value_host);
tt_status tt_l2_norm_f64(tt_handle *h, const double *c_dev, double *grad_dev, double *value_host);
tt_status tt_tv_huber(tt_handle *h, const float *c_dev, double delta, float *grad_dev, double *value_host);
tt_status tt_tv_huber_f64(tt_handle *h, const double *c_dev, double delta, double *grad_dev, double *value_host);

/* L-BFGS (Section "Optimization"), unbounded two-loop recursion with memory
 * m and backtracking Armijo line search (c1 = 1e-4, step halving, at most 20
 * evaluations per iteration; first iteration steps 1/|g| along -g; a pair is
 * stored only if s.y > 1e-10 |s||y|; a non-descent direction clears the
 * memory).  Vectors live on the device in the handle's precision.  The
 * two loops run on the FP64 Gram matrix of the stored pairs and the gradient
 * (the same recursion in exact arithmetic; three vector kernels per
 * iteration); dot products of float vectors use compensated FP32 (Dot2)
 * accumulation within a CTA and FP64 across CTAs.  I_dev / W_dev (W may be NULL) are
 * referenced, not copied: keep them alive and unchanged while the state
 * exists.  tt_lbfgs_create evaluates the loss and gradient at c0_dev;
 * c0_dev may be NULL to start at zero (that evaluation then skips the
 * forward projection, as tt_gradient_residual does for c_dev == NULL). */
tt_status tt_lbfgs_create(tt_handle *h, int m, const void *c0_dev, const void *I_dev,
                          const void *W_dev, tt_lbfgs **out);
/* A state started at the minimiser of the loss (Section "Optimization")
 * along the ray {a u_dev}, at the cost of ONE gradient evaluation, the one
 * at u_dev: the learned warm start scales the network's output u_dev this
 * way (the paper has no warm start; this entry point serves it).  g0_dev and loss0 are the gradient and loss
 * at zero from an earlier evaluation (tt_gradient_residual at c = 0,
 * g0 = -2 A^T W I, loss0 = sum W I^2).  The loss is quadratic along the ray,
 * L(a u) = a^2 |A u|^2_W - 2 a <A u, W I> + loss0, with <A u, W I> =
 * -<u, g0>/2 and |A u|^2_W = L(u) - loss0 + 2 <A u, W I>; the state starts at
 * a* u, a* = <A u, W I> / |A u|^2_W, with loss loss0 - <A u, W I>^2 / |A u|^2_W
 * and gradient a* g(u) + (1 - a*) g0 (no evaluation at a* u).  If the ray
 * does not lower the loss (A u = 0, or a non-finite value), the state starts
 * at zero with (loss0, g0) and *alpha_out = 0.  *alpha_out (may be NULL)
 * receives a*.  u_dev and g0_dev: [nx][ny][nz][K], the handle's API type,
 * 16-byte aligned, read only; I_dev / W_dev as for tt_lbfgs_create.  The
 * state's evaluation counter starts at 1 (the evaluation at u).  On a
 * handle with 2-byte volume storage (TT_BF16, TT_F16) the evaluation rounds
 * the volume it projects, so the start's loss and gradient differ from an
 * evaluation at a* u by that rounding (relative 2^-9 / 2^-12 of the A u
 * terms), as every result of such a handle does.  Returns TT_INVALID_ARG for
 * a bad argument, TT_NONFINITE if L(u) is not finite. */
tt_status tt_lbfgs_create_ray(tt_handle *h, int m, const void *u_dev, const void *g0_dev, double loss0,
                              const void *I_dev, const void *W_dev, double *alpha_out, tt_lbfgs **out);
/* One iteration.  c_out_dev (may be NULL) receives the new iterate
 * [nx][ny][nz][K]; *loss_host the new loss; *n_evals_host the number of
 * gradient evaluations used.  On TT_LINESEARCH_FAILED the iterate is
 * unchanged. */
tt_status tt_lbfgs_step(tt_handle *h, tt_lbfgs *st, void *c_out_dev, double *loss_host,
                        int *n_evals_host);
/* Current iterate / gradient / loss of the state. */
tt_status tt_lbfgs_get(tt_handle *h, tt_lbfgs *st, void *c_dev, void *g_dev, double *loss_host);
/* Frees the state; valid before or after tt_destroy of its handle. */
tt_status tt_lbfgs_destroy(tt_lbfgs *st);
/* Counters of the state (any pointer may be NULL): accepted iterations,
 * gradient evaluations including the one of tt_lbfgs_create, and the
 * line-search step a of the last accepted iteration (x_new = x + a d; a = 1
 * is the full quasi-Newton step; with no stored pairs d = -g and the search
 * starts at a = 1/|g|). */
tt_status tt_lbfgs_stats(const tt_lbfgs *st, long long *iterations, long long *evaluations, double *last_step);
/* Checkpoint / resume of an L-BFGS state.  tt_lbfgs_checkpoint_bytes gives
 * the size of the state's checkpoint as it stands (it grows with the number
 * of stored pairs; 0 for NULL).  tt_lbfgs_save writes it into the host
 * buffer buf (at least that many bytes; caller-owned, any host memory) and
 * synchronises the handle's stream: a header (magic "TTLBFGS1", memory m,
 * stored pairs, newest slot, element size, n, loss, the counters of
 * tt_lbfgs_stats), the FP64 Gram matrix, then the iterate, the gradient and
 * the stored pairs, newest first, as n-element vectors of the handle's
 * element type.  tt_lbfgs_restore creates
 * a state of handle h from such a buffer (bytes = its exact size); I_dev /
 * W_dev are not part of a checkpoint and are passed as to tt_lbfgs_create.
 * The restored state continues exactly as the saved one would have.
 * Errors: TT_INVALID_ARG for a buffer that is too small, not a checkpoint,
 * or one of another problem size or precision. */
long long tt_lbfgs_checkpoint_bytes(const tt_lbfgs *st);
tt_status tt_lbfgs_save(tt_handle *h, const tt_lbfgs *st, void *buf, long long bytes);
tt_status tt_lbfgs_restore(tt_handle *h, const void *buf, long long bytes, const void *I_dev,
                           const void *W_dev, tt_lbfgs **out);

/* ---- SIRT-preconditioned solver (Section "Standard reconstruction
 * pipelines": SIRT as preconditioned gradient descent on weighted least
 * squares, the same weights applied to the full model A = B_s (x) P_s, and
 * Nesterov momentum).  The paper gives no formulas; the weights are built
 * from |A| = |B_s| (x) P_s (the John-transform coefficients are >= 0):
 *   rho[s][j][k][c] = (sum_i |B_s[c][i]|) (P_s 1)[j][k]        row sums of |A|
 *   kappa[v][i]     = sum_s (sum_c |B_s[c][i]|) (P_s^T 1)[v]  column sums
 *   R = W / rho (0 on rays whose length in the volume is <= 1e-6 a)
 *   D = 1 / kappa (0 where kappa <= 1e-6 a / (2 sqrt(pi)))
 * With 0 <= W <= 1, ||R^1/2 A D^1/2||_2 <= 1 (Cauchy-Schwarz), so the
 * iteration below is stable for 0 < eta < 2.
 *
 * tt_sirt_weights: R_dev [S][nj][nk][C] and D_dev [nx][ny][nz][K] (caller
 * allocated, 16-byte aligned, handle precision's API type) from the
 * optional data weights W_dev (NULL = 1).  Runs the projector kernels on a
 * unit volume, so it overwrites the handle's internal buffers (not the
 * caller's).  Asynchronous on the handle's stream. */
tt_status tt_sirt_weights(tt_handle *h, const float *W_dev, float *R_dev, float *D_dev);
tt_status tt_sirt_weights_f64(tt_handle *h, const double *W_dev, double *R_dev, double *D_dev);
/* Solver state for minimising L_R(c) = sum R (A c - I)^2 by
 *   y_t = x_t + mu_t (x_t - x_{t-1}),   x_{t+1} = y_t - (eta/2) D grad L_R(y_t)
 * (x_1 = x_0 = c0; eta = 1, momentum = 0 is the classical SIRT update
 * x + D A^T R (I - A x)).  momentum < 0 selects the Nesterov schedule
 * mu_t = (t-1)/(t+2); otherwise mu_t = momentum.  Needs 0 < eta < 2 and
 * momentum < 1 (else TT_INVALID_ARG).  c0_dev and W_dev are copied (the
 * weights into R); I_dev [S][nj][nk][C] must stay valid for the state's
 * life.  Pointers are device pointers of the handle's API type. */
tt_status tt_mitra_create(tt_handle *h, const void *c0_dev, const void *I_dev, const void *W_dev,
                          double eta, double momentum, tt_mitra **out);
/* One iteration: one gradient-residual evaluation at y_t and one update
 * kernel.  loss_host (may be NULL) receives L_R(y_t): the call returns as
 * soon as the adjoint has published that loss, with the rest of the adjoint
 * and the update kernel still in flight (x and y are stream-ordered outputs,
 * like every device result).  With NULL the call only enqueues work (no host
 * synchronisation). */
tt_status tt_mitra_step(tt_mitra *m, double *loss_host);
/* Copies the iterate x (c_dev, [nx][ny][nz][K]), the data weights R
 * (R_dev) and the preconditioner D (D_dev); any may be NULL.  *iterations
 * (may be NULL) = iterations taken. */
tt_status tt_mitra_get(tt_mitra *m, void *c_dev, void *R_dev, void *D_dev, int *iterations);
/* Frees the state; valid before or after tt_destroy of its handle. */
tt_status tt_mitra_destroy(tt_mitra *m);

/* Learned warm start: a 3-D convolutional network (4 layers of 3x3x3
 * convolutions, k_in -> 32 -> 32 -> 32 -> k_out channels, ReLU between
 * layers, no biases; "same" zero padding) that maps the first back-projected
 * gradient of a reconstruction to a starting coefficient volume.  The paper's
 * outlook proposes simulated data for training machine-learning models; the
 * network and its training are this library's.  Weights are kept in FP32
 * (Adam), activations in bfloat16, convolutions run on the tensor cores with
 * FP32 accumulation.  Volumes are [nx][ny][nz][channels] FP32 device arrays.
 * Because the network is bias-free and ReLU is positively homogeneous,
 * y = out_scale * net(x / in_scale) is exactly equivariant to the scale of x.
 *   w_host: HOST array of tt_wsnet_num_weights(k_in, k_out) floats, layer by
 *   layer, each [3][3][3][c_out][c_in] (tap index (dx+1, dy+1, dz+1)).
 *   tt_wsnet_forward:    y = out_scale * net(x / in_scale).
 *   tt_wsnet_gradient:   loss = mean((net(x/in_scale) - target/out_scale)^2) over
 *                        voxels and k_out channels, and its weight gradient
 *                        into grad_host (may be NULL); synchronises.
 *   tt_wsnet_train_step: the same loss, then one Adam step (beta 0.9, 0.999,
 *                        eps 1e-8, learning rate lr); synchronises. */
typedef struct tt_wsnet tt_wsnet;
int tt_wsnet_num_weights(int k_in, int k_out);
tt_status tt_wsnet_create(int k_in, int k_out, const float *w_host, void *stream, tt_wsnet **out);
tt_status tt_wsnet_destroy(tt_wsnet *net);
tt_status tt_wsnet_set_stream(tt_wsnet *net, void *stream);
tt_status tt_wsnet_forward(tt_wsnet *net, int nx, int ny, int nz, const float *x_dev, double in_scale,
                           double out_scale, float *y_dev);
tt_status tt_wsnet_gradient(tt_wsnet *net, int nx, int ny, int nz, const float *x_dev, const float *target_dev,
                            double in_scale, double out_scale, float *grad_host, double *loss_host);
tt_status tt_wsnet_train_step(tt_wsnet *net, int nx, int ny, int nz, const float *x_dev, const float *target_dev,
                              double in_scale, double out_scale, double lr, double *loss_host);
tt_status tt_wsnet_get_weights(tt_wsnet *net, float *w_host);
/* The network's two convolution kernels on their own (bfloat16 operands as
 * raw 16-bit words, device pointers, enqueued on stream):
 *   tt_conv3d_bf16:       y[v][co] = sum_t sum_ci x[v + d_t][ci] w[t][co][ci]
 *                         (x [nvox][cin], w [27][cout][cin], y float [nvox][cout];
 *                         relu must be 0);
 *   tt_conv3d_wgrad_bf16: dw[t][co][ci] += sum_v dy[v][co] x[v + d_t][ci]
 *                         (dy [nvox][cout], dw float [27][cout][cin]).
 * cin, cout in {16, 32}. */
tt_status tt_conv3d_bf16(int nx, int ny, int nz, int cin, int cout, const void *x_dev, const void *w_dev, int relu,
                         float *y_dev, void *stream);
/* The network's hidden-layer form of the same convolution: y_dev bfloat16
 * [nvox][cout] (raw 16-bit words), the FP32 accumulation with ReLU (relu !=
 * 0) rounded once to bfloat16.  Compiled for (cin, cout) = (16, 32) and
 * (32, 32), and without ReLU also (32, 16); other pairs: TT_UNSUPPORTED. */
tt_status tt_conv3d_bf16_act(int nx, int ny, int nz, int cin, int cout, const void *x_dev, const void *w_dev,
                             int relu, void *y_dev, void *stream);
tt_status tt_conv3d_wgrad_bf16(int nx, int ny, int nz, int cin, int cout, const void *x_dev, const void *dy_dev,
                               float *dw_dev, void *stream);

/* One 128 x N tile on the tcgen05 tensor cores (the building block of the
 * warm start's convolutions; the paper has no counterpart): C = A B^T with
 * A_dev [128][K] and B_dev [N][K] bfloat16 row-major, C_dev [128][N] float,
 * all device memory.  N and K multiples of 16 in [16, 256].  One CTA on
 * stream; *status_dev (device int) is set to 0, or to 1 when the wait for
 * the tensor cores gave up (results then unset). */
tt_status tt_umma_gemm_bf16(const void *A_dev, const void *B_dev, float *C_dev, int N, int K, int *status_dev,
                            void *stream);

/* Phantom helper: SH coefficients of zonal functions rotated to unit axes n,
 * c_lm = a_l sqrt(4 pi/(2l+1)) Y_lm(n) (addition theorem).  dirs_dev [n][3],
 * amps_dev [n][ell_max/2+1], c_dev [n][K], FP32, device, on stream. */
tt_status tt_zonal_to_sh(int ell_max, long long n, const float *dirs_dev, const float *amps_dev,
                         float *c_dev, void *stream);

/* Kernel-time accounting.  When enabled, every kernel libtt launches on the
 * handle's stream is bracketed by CUDA events (the launches of one gradient
 * evaluation, enqueued back to back, share their boundary events, so a
 * launch's time includes the gap before the next one); tt_profile_enable
 * pre-creates the events, and completed pairs are recycled as later launches
 * are enqueued.  tt_profile_read synchronises and returns, for kernel class
 * `slot`, the summed device time in ms and the launch count since the last
 * reset.  tt_launch_count counts all kernel launches of the handle since
 * creation (always on). */
enum {
    TT_KSLOT_PACK = 0, TT_KSLOT_FORWARD = 1, TT_KSLOT_BACKCONTRACT = 2, TT_KSLOT_ADJOINT = 3,
    TT_KSLOT_UNPACK = 4, TT_KSLOT_REDUCE = 5, TT_KSLOT_BASIS = 6, TT_KSLOT_VECTOR = 7,
    TT_KSLOT_COUNT = 8
};
tt_status tt_profile_enable(tt_handle *h, int enable);
tt_status tt_profile_read(tt_handle *h, int slot, double *total_ms, long long *launches);
tt_status tt_profile_reset(tt_handle *h);
const char *tt_kernel_slot_name(int slot);
long long tt_launch_count(const tt_handle *h);

#ifdef __cplusplus
}
#endif
#endif /* TT_H */
