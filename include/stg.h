/*
 * stg.h -- C ABI of the GB300 space-time Vanka-multigrid FGMRES solver.
 *
 * The solver follows M. Anselmann, M. Bause, "Efficiency of local Vanka smoother
 * geometric multigrid preconditioning for space-time finite element methods to
 * the Navier--Stokes equations":
 *   - Sec. 2, Eq. (2.2): the dG(k)-in-time, (Q2)^d x P1disc-in-space slab problem
 *     on I_n with Nitsche's method for Dirichlet data (Eq. (2.1));
 *   - Sec. 3, Eq. (3.2): the unknown X_n = (v^{n,0}, p^{n,0}, ..., v^{n,k}, p^{n,k})
 *     of the k+1 Gauss--Radau time nodes;
 *   - Sec. 3, Eq. (3.3): the Newton/Oseen Jacobian J_n with (k+1) x (k+1)
 *     saddle-point blocks [[D_ab, B_ab^T], [B_ab, 0]];
 *   - Sec. 3: GMRES preconditioned by one geometric-multigrid V-cycle, a direct
 *     solver on the coarsest mesh T_0 and the local Vanka smoother
 *     S_K(d) = R_K d + omega J_K^{-1} R_K (b - J d) (Eq. (3.4)) applied through
 *     the averaging loop (S0)-(S3).
 *
 * Conventions shared by every entry point:
 *   - Vectors are caller-owned DEVICE buffers of doubles (e.g. torch tensors) in
 *     the C-ABI order of X_n: time-node blocks a = 0..k; inside block a the R
 *     velocity values (Q2 nodes numbered lexicographically with x fastest,
 *     components interleaved: node*d + c), then the S pressure values (cells
 *     numbered lexicographically with x fastest, d+1 P1disc coefficients
 *     {1, xi_1, .., xi_d} per cell in the cell's reference coordinates).
 *     Internally the library permutes to its own layout.
 *   - All work is ordered on the stream given to stg_setup; entry points that
 *     return scalars to the host synchronise that stream.  stg_setup and
 *     stg_update_linearisation fork part of their work (the coarse factorisation,
 *     the intermediate levels) onto two higher-priority streams the context owns
 *     and join them back into the given stream before they return.
 *   - Errors are returned as a status; no call aborts.  stg_last_error gives a
 *     text.  The context stays usable after STG_ENOCONV and STG_ESINGULAR.
 *   - The context owns all device memory it allocates (freed by stg_destroy).
 */
#ifndef STG_H
#define STG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stg_ctx stg_ctx;

typedef enum {
  STG_OK = 0,
  STG_EINVAL = 1,     /* invalid argument (sizes, levels, null pointers)            */
  STG_ENOMEM = 2,     /* device allocation failed                                    */
  STG_ECUDA = 3,      /* a CUDA call or kernel launch failed                         */
  STG_ESINGULAR = 4,  /* a zero pivot in a local J_K or a coarse block (cell id in   */
                      /* stg_last_error)                                            */
  STG_ENOCONV = 5,    /* FGMRES reached gmres_maxit; x and rel_res are still written */
  STG_ETIMEOUT = 6    /* a device-side wait reached its iteration limit              */
} stg_status;

enum { STG_OSEEN = 0, STG_NEWTON = 1 };                 /* Sec. 3: terms of D_ab        */
enum { STG_VANKA_AVERAGED = 0, STG_VANKA_COLOURED = 1 }; /* (S0)-(S3) / successive       */
enum { STG_F64 = 0, STG_F32 = 1, STG_BF16 = 2 };        /* storage/arithmetic precision */

/* Structured box mesh hierarchy (Sec. 2: nested partitions T_0..T_L, h_l = h_{l-1}/2).
 * nx, ny (, nz) are the FINEST level's cells per direction; level l has
 * n/2^(n_levels-1-l) cells per direction, so every n must be divisible by
 * 2^(n_levels-1).  Bit 2*dir+side of dirichlet_faces marks a Dirichlet face
 * (side 0 = low, 1 = high); the other faces carry the do-nothing condition
 * (Sec. 1).
 * obstacle (2D only): the cells [obstacle[0], obstacle[1]) x [obstacle[2],
 * obstacle[3]) of the COARSEST level (and their children on every finer level)
 * are removed from the domain, a structured stand-in for the obstacle of the
 * benchmark of Sec. 4; the faces of the remaining cells that border it carry
 * Dirichlet data (Nitsche's method, Eq. (2.1)).  The unknowns left without an
 * equation (velocity at Q2 nodes of removed cells only, pressure of removed
 * cells) keep their place in the vectors with identity rows; solutions are zero
 * there for zero right-hand sides.  All four zero: no obstacle. */
typedef struct {
  int dim;                 /* 2 or 3 */
  int nx, ny, nz;          /* finest-level cells (nz ignored for dim = 2) */
  int n_levels;            /* >= 1; level 0 is solved directly */
  double x0, x1, y0, y1, z0, z1;
  unsigned dirichlet_faces;
  int obstacle[4];         /* x_lo, x_hi, y_lo, y_hi in coarsest-level cells (2D)  */
  int order;               /* velocity order r of (Q_r)^d x P_{r-1}^disc (Sec. 2): 2    */
                           /* (0 also means 2) or 4 (2D, k <= 2, no obstacle; the pair */
                           /* of the paper's 2D experiment).  Q_r nodes: r n + 1 per   */
                           /* direction; P_{r-1}^disc: the monomials of total degree   */
                           /* <= r - 1 in the cell's reference coordinates, ordered by */
                           /* degree and then with the x exponent falling (r = 2:      */
                           /* {1, xi, eta}; r = 4: 10 coefficients).  Newton, the warm */
                           /* start and the drag/lift entry points need order 2.       */
} stg_mesh;

typedef struct {
  int linearisation;       /* STG_NEWTON (default) adds ((v . grad) w, psi) to D_ab   */
  int smoother;            /* STG_VANKA_AVERAGED (default, (S0)-(S3)) | COLOURED     */
  int nu1, nu2;            /* pre/post smoothing steps J_max (paper: 4; default 4)   */
  double omega;            /* under-relaxation of Eq. (3.4) (paper: 0.7)             */
  double gamma1, gamma2;   /* Nitsche penalties of Eq. (2.1) (paper: 35, 35)         */
  int factor_prec;         /* storage of J_K^{-1}: STG_F64 | STG_F32 | STG_BF16       */
  int vcycle_prec;         /* vectors/operators inside the V-cycle: STG_F64 | STG_F32 */
  int gmres_restart;       /* FGMRES restart length (default 30)                      */
  int gmres_maxit;         /* total inner iterations (default 200)                    */
  double gmres_rtol;       /* stop at ||b - J x|| <= max(rtol ||b||, atol)            */
  double gmres_atol;       /* (defaults 1e-8 and 0; the paper's absolute 1e-9: set    */
                           /*  rtol = 0, atol = 1e-9)                                  */
  int use_graph;           /* capture the V-cycle in a CUDA graph (default 1)         */
  int coarse_refine;       /* steps of iterative refinement with FP64 residuals      */
                           /* after each coarse solve (default 1): with FP32 coarse   */
                           /* factors, and in the FP64 V-cycle (whose explicit block  */
                           /* inverses it brings to the accuracy of an LU solve)      */
  int coarse_prec;         /* FP32 V-cycle only: precision of the coarse factors,     */
                           /* STG_F32 (default; refined as above) or STG_F64 (one    */
                           /* FP64 solve per cycle, no refinement, but an FP64       */
                           /* factorisation ~20x slower on GB300); the FP64 V-cycle  */
                           /* always uses FP64 coarse factors                         */
  int overlap_launches;    /* 1 (default): the V-cycle's kernels are launched with    */
                           /* programmatic dependent launch, so each launch may begin */
                           /* before its predecessor is retired; every such kernel    */
                           /* waits for its predecessor's completion before touching  */
                           /* memory, so results are identical with 0.  Not applied   */
                           /* inside the branches of a stg_batch graph.               */
} stg_options;

/* Fills the defaults listed above.  Returns STG_EINVAL for a null pointer. */
stg_status stg_options_default(stg_options* opt);

/* Builds the level hierarchy, assembles J_l on every level (Eq. (3.3); coarse
 * operators rediscretised with w injected at the coarse Q2 nodes), inverts
 * every local J_K on levels l >= 1 (Eq. (3.4)) and factors J_0.
 *   k      dG(k) degree, 0 <= k <= 4 (dim 2) or 0 <= k <= 2 (dim 3)
 *   nu     viscosity; tau the slab length t_n - t_{n-1}
 *   w      DEVICE doubles [(k+1) * R]: the linearisation velocity at the Q2
 *          nodes of the finest level for each Radau node, in the velocity
 *          part of the C-ABI order (block a holds R values); read during the
 *          call only, caller-owned
 *   stream a cudaStream_t (NULL = legacy default stream)
 *   out    receives the new context (NULL on failure)
 * Returns STG_EINVAL (bad mesh/k/options), STG_ENOMEM, STG_ECUDA or
 * STG_ESINGULAR (a local J_K or the coarse system has a zero pivot). */
stg_status stg_setup(const stg_mesh* mesh, int k, double nu, double tau, const double* w,
                     const stg_options* opt, void* stream, stg_ctx** out);

/* Re-assembles and re-factors every level for a new linearisation velocity w
 * (same layout as in stg_setup); allocates nothing. */
stg_status stg_update_linearisation(stg_ctx* ctx, const double* w);

/* Changes the slab length tau = t_n - t_{n-1} of the context (Sec. 4 marches with
 * tau_n = 0.1, 0.05, 0.01; Eq. (2.2) integrates every spatial term of slab I_n with
 * the weights tau w_a).  Re-assembles the w-independent part of every level and
 * re-linearises every level at the current linearisation velocity (the last one
 * given to stg_setup / stg_update_linearisation, or the last Newton iterate after
 * stg_newton_slab); allocates nothing.  tau must be finite and >= 0 (STG_EINVAL
 * otherwise).  tau = 0 leaves every local J_K without its pressure coupling and
 * returns STG_ESINGULAR with the cell id in stg_last_error; the context stays
 * usable and a later call with tau > 0 restores it. */
stg_status stg_set_slab_length(stg_ctx* ctx, double tau);

/* y = J x on the finest level (Eq. (3.3)); x, y DEVICE doubles of length N. */
stg_status stg_apply_jacobian(stg_ctx* ctx, const double* x, double* y);

/* y = J_l x on level `level` (0 = coarsest); vectors in that level's C-ABI order. */
stg_status stg_apply_level_jacobian(stg_ctx* ctx, int level, const double* x, double* y);

/* x = V(b): one V-cycle on the finest level with initial guess 0 (Sec. 3),
 * nu1 pre- and nu2 post-smoothing steps on levels >= 1, the direct solve on
 * level 0.  b, x DEVICE doubles of length N. */
stg_status stg_vcycle(stg_ctx* ctx, const double* b, double* x);

/* `sweeps` smoothing steps on level `level` >= 1 for J_l x = b, updating x in
 * place ((S0)-(S3) for STG_VANKA_AVERAGED).  Runs in the V-cycle precision. */
stg_status stg_smooth(stg_ctx* ctx, int level, int sweeps, const double* b, double* x);

/* Grid transfer (nested FE spaces; time nodes are not coarsened):
 * stg_prolongate: x_fine += P x_coarse; stg_restrict: b_coarse = P^T r_fine.
 * `level` is the FINE level (>= 1); vectors in the levels' C-ABI orders. */
stg_status stg_prolongate(stg_ctx* ctx, int level, const double* x_coarse, double* x_fine);
stg_status stg_restrict(stg_ctx* ctx, int level, const double* r_fine, double* b_coarse);

/* x = J_0^{-1} b on the coarsest level (Sec. 3: direct solver on T_0).  With
 * Dirichlet data on the whole boundary J_0 is singular (one constant-pressure
 * mode per Radau node); the solution then has the pressure coefficient 0 of
 * cell 0 equal to 0 for every Radau node.  b must be consistent. */
stg_status stg_coarse_solve(stg_ctx* ctx, const double* b, double* x);

/* Flexible GMRES, right-preconditioned by one V-cycle (Sec. 3).  x holds the
 * initial guess on entry and the solution on exit; iters (total inner
 * iterations) and rel_res (||b - J x|| / ||b||, recomputed in FP64) are host
 * pointers, may be NULL, and are written even on STG_ENOCONV. */
stg_status stg_gmres_solve(stg_ctx* ctx, const double* b, double* x, int* iters, double* rel_res);

/* Damped Newton for the nonlinear slab problem F_n(X_n) = 0 of Eq. (3.2)
 * (Sec. 3): F_n(X) = J_Oseen(w = v(X)) X - b with
 *   b_a = tau w_a [ (f_a, psi) + B_GammaD(g_a, (psi, xi)) ] + chi_a(0) (v_prev, psi),
 * each correction from J_Newton(v(X)) C = -F_n(X) by FGMRES with the V-cycle
 * (options of the context), damping lambda = 1, 1/2, .., 1/16 until
 * ||F(X + lambda C)|| < (1 - 1e-4 lambda) ||F(X)|| (1/16 is taken otherwise).
 *   v_prev  DEVICE [R] velocity at t_{n-1} (velocity part of the C-ABI order) or NULL (0)
 *   f, g    DEVICE [(k+1) R] body force and Dirichlet data at the finest Q2 nodes per
 *           Radau node (the integrals use their Q2 interpolants) or NULL (0)
 *   X       DEVICE [N]: initial guess in, solution out (C-ABI order)
 *   stops when ||F|| <= max(rtol ||F(X_0)||, atol) or after maxit steps (STG_ENOCONV)
 * newton_steps, gmres_iters (total), residual (final ||F||) are host pointers, may be
 * NULL.  Afterwards the finest operator holds the Oseen Jacobian of the final iterate and
 * the other levels the Newton Jacobian of the previous one: call
 * stg_update_linearisation before using the linear-solve entry points again. */
stg_status stg_newton_slab(stg_ctx* ctx, const double* v_prev, const double* f, const double* g, double* X,
                           double rtol, double atol, int maxit, int* newton_steps, int* gmres_iters,
                           double* residual);

/* Drag and lift (Sec. 4 reports drag and lift coefficients of the flow around the
 * obstacle, from surface integrals of the stress): the force of the fluid on the
 * obstacle of the mesh at every Radau node a of slab vector X (DEVICE, C-ABI order),
 *   F_a = - int_S (nu grad v_h - p_h I) n dS,
 * S the obstacle's faces, n the unit normal of the fluid domain (pointing into the
 * obstacle), v_h and p_h from the fluid cells next to S, 3-point Gauss rule per face.
 * forces: HOST doubles [k+1][2] = (F_x, F_y) per Radau node (drag, lift; the
 * coefficients are 2 F / (U_mean^2 D)).  STG_EINVAL without an obstacle. */
stg_status stg_obstacle_forces(stg_ctx* ctx, const double* X, double* forces);

/* X0 = the previous slab's end value (the last Radau-node block of X_prev, velocity
 * and pressure) repeated at every Radau node: the initial guess of the next slab.
 * DEVICE vectors of length N in the C-ABI order. */
stg_status stg_slab_initial_guess(stg_ctx* ctx, const double* X_prev, double* X0);

/* Sizes of level `level`: space-time DoFs N_l = (k+1)(R+S), cells, and the
 * local patch size (k+1)(R^ + S^) (21(k+1) in 2D, 85(k+1) in 3D).  Host
 * pointers, each may be NULL. */
stg_status stg_get_sizes(const stg_ctx* ctx, int level, long long* n_dofs, long long* n_cells,
                         int* n_patch);

/* Copies J_K^{-1} of cell `cell` (cell number as in the C-ABI order) of level
 * `level` >= 1 to the HOST buffer out[n_patch * n_patch], row-major, in the
 * paper's local order dof(K, mu): time node a first, then the 3^d Q2 nodes
 * (x fastest) times d components, then the d+1 pressure coefficients.  The
 * values are those stored for the smoother (rounded to factor_prec). */
stg_status stg_get_local_inverse(const stg_ctx* ctx, int level, long long cell, double* out);

/* Instrumentation.  stg_profile(ctx, 1) records CUDA events on the context's
 * stream around the launches of the smoother's colour kernel on the finest
 * level (y_K = J_K^{-1} R_K r for the cells of one colour, Eq. (3.4)) in one
 * sweep per V-cycle (the last post-smoothing sweep, or the last pre-smoothing
 * sweep when nu2 = 0; the last sweep of stg_smooth) and accumulates their
 * device time; stg_profile(ctx, 0) stops and resets.  The
 * V-cycle graph is recaptured when the setting changes.  stg_profile_read
 * returns the accumulated milliseconds, the number of launches and the number
 * of patches they processed (host pointers, each may be NULL). */
stg_status stg_profile(stg_ctx* ctx, int enable);
stg_status stg_profile_read(const stg_ctx* ctx, double* total_ms, long long* launches, long long* patches);

/* Number of kernels this library has enqueued in this process (a CUDA-graph
 * replay counts each of its kernel nodes). */
long long stg_kernel_launches(void);

/* Allocation-free batched inverse of caller-supplied dense matrices.  (The
 * paper has no counterpart: it is a service for callers that cannot allocate
 * device memory when they need local inverses -- host applications that own
 * the GPU's memory and hand it out only from their own pools or arenas, and
 * real-time loops that forbid cudaMalloc/cudaFree after start-up because those
 * calls may synchronise the device and take unbounded time.)
 *   n       matrix order, 1 <= n <= 256 (else STG_EINVAL with a message)
 *   count   number of matrices (0 is a no-op)
 *   a       DEVICE doubles [count][n][n], row-major, caller-owned, read only
 *   a_inv   DEVICE doubles [count][n][n], row-major, caller-owned: the inverses
 *           (Gauss-Jordan with partial pivoting), zeros for a singular matrix
 *   stream  cudaStream_t for the work; the call synchronises it
 * Needs no context and allocates nothing: the working copies live in one
 * 8 MiB array compiled into the library (2^20 doubles, so one launch takes
 * at most 2^20 / n^2 matrices and larger counts run in several launches),
 * which every GPU that loads the library holds until the process exits.  The
 * first call on a device looks up that array's device address.  All calls
 * share the array and keep the last call's contents, so calls that overlap on
 * the GPU (other streams or host threads) race.  Returns STG_ESINGULAR (the
 * lowest index of a matrix with a zero pivot in stg_last_error(NULL)) or
 * STG_ECUDA on failure. */
stg_status stg_invert_local_noalloc(int n, long long count, const double* a, double* a_inv, void* stream);

/* Autotuner: times every variant of the smoother's colour kernel (one warp per
 * patch: 3 column-batch depths x 3 CTA sizes; factors staged in shared memory by
 * bulk copies: 4 pipeline shapes) on every level >= 1 and keeps the fastest per level; the
 * V-cycle graph is recaptured.  variant (host, may be NULL) receives the finest
 * level's choice, sweep_ms (host, may be NULL) the finest level's time of one
 * sweep's colour kernels.  (Engineering service; the paper has no counterpart.) */
stg_status stg_autotune(stg_ctx* ctx, int* variant, double* sweep_ms);

/* Fault-injection hook for the bounded waits (engineering service): sets the
 * iteration limit with which the staged smoother kernels wait for a factor
 * copy (default 2^22; the value applies to every context of the process and to
 * captured graphs).  A kernel that reaches the limit lets its copies in flight
 * land, returns, and the next synchronising call of the context reports
 * STG_ETIMEOUT; 0 makes every such wait give up at once.  STG_EINVAL for a
 * negative limit. */
stg_status stg_set_wait_limit(long long spins);

/* Colour-kernel variant of level `level` >= 1 (0..16, as timed by stg_autotune):
 * read it, or set it (the V-cycle graph is recaptured), e.g. to replay a choice
 * made in another run.  STG_EINVAL for a level or variant out of range. */
stg_status stg_get_colour_variant(const stg_ctx* ctx, int level, int* variant);
stg_status stg_set_colour_variant(stg_ctx* ctx, int level, int variant);

/* Batched solves of several independent problems (contexts of any mesh size and
 * k, each created with a non-default stream; contexts may share one): the
 * V-cycles of all problems are captured once into a single CUDA graph with one
 * concurrent branch per problem, and stg_batch_gmres_solve runs FGMRES (Sec. 3) on all problems in lock
 * step, one graph launch per iteration.  b, x: HOST arrays of n DEVICE pointers
 * (C-ABI order of each problem); iters, rel: host arrays of n entries or NULL.
 * The contexts must not be used elsewhere while they belong to a batch, and the
 * batch must be destroyed before them.  (The paper has no counterpart.) */
typedef struct stg_batch stg_batch;
stg_status stg_batch_create(int n, stg_ctx* const* ctxs, stg_batch** out);
stg_status stg_batch_gmres_solve(stg_batch* batch, const double* const* b, double* const* x, int* iters,
                                 double* rel);
void stg_batch_destroy(stg_batch* batch);

/* ------------------------------------------------------------------------
 * Learned warm start of the next time slab.  The paper has no learned part: it
 * time-marches slab problems (Eq. (2.2)) and solves each by Newton (Sec. 3),
 * and the Newton iteration needs an initial guess X^0 for slab n+1.  The
 * fallback is stg_slab_initial_guess (slab n's end value at every Radau node).
 * Here a small convolutional network, trained on the slabs the solver itself
 * produced, predicts the part of slab n+1's velocity that linear extrapolation
 * from the end values of slabs n-1 and n misses.
 *
 * Network: L = n_layers 3x3 convolutions, zero padding, with bias, tanh after
 * every layer but the last:
 *   y[b][o][i][j] = bias[o] + sum_{c,dy,dx} w[o][c][dy][dx] x[b][c][i+dy-1][j+dx-1].
 * Tensors are FP32 NCHW arrays in DEVICE memory: [batch][channels][height][width].
 * Parameters: one flat FP32 array, per layer w[c_out][c_in][3][3] then bias[c_out].
 * Loss: mean of (y - t)^2 over all batch * c_L * height * width outputs.
 * Training: Adam (Kingma & Ba) with beta1 = 0.9, beta2 = 0.999, eps = 1e-8.
 * All work runs on the stream given at creation; the network object owns its
 * buffers and must not be used from two host threads at once.
 * ------------------------------------------------------------------------ */
typedef struct stg_cnn stg_cnn;
typedef struct {
  int n_layers;      /* 1..8 */
  int channels[9];   /* channels[0] = input, channels[n_layers] = output; each 1..32 */
  int height, width; /* image size */
  int max_batch;     /* largest batch of any later call */
} stg_cnn_desc;

/* Creates the network with all parameters zero.  stream: cudaStream_t.
 * STG_EINVAL for a bad descriptor, STG_ENOMEM when device memory runs out. */
stg_status stg_cnn_create(const stg_cnn_desc* desc, void* stream, stg_cnn** out);
/* Number of FP32 parameters (host output). */
stg_status stg_cnn_n_params(const stg_cnn* net, long long* count);
/* Copies all parameters from / to a HOST array of stg_cnn_n_params floats; set also
 * resets the Adam moments and step count.  Both synchronise the stream. */
stg_status stg_cnn_set_params(stg_cnn* net, const float* params);
stg_status stg_cnn_get_params(stg_cnn* net, float* params);
/* y[batch][c_L][H][W] = network(x[batch][c_0][H][W]); device pointers; asynchronous. */
stg_status stg_cnn_forward(stg_cnn* net, const float* x, float* y, int batch);
/* Gradient of the loss for input x and target t (device, [batch][c_L][H][W]) with
 * respect to all parameters into grad (device, n_params floats, same layout as the
 * parameters); loss (host, may be NULL) receives the loss, which synchronises. */
stg_status stg_cnn_gradients(stg_cnn* net, const float* x, const float* t, int batch, float* grad, double* loss);
/* One Adam update of the parameters with gradient grad (device). */
stg_status stg_cnn_adam_step(stg_cnn* net, const float* grad, float lr, float beta1, float beta2, float eps);
/* n_steps Adam steps with learning rate lr; step s uses the samples
 * order[s*batch .. s*batch + batch-1] (HOST ints in [0, n_samples)) of the device
 * arrays x_all[n_samples][c_0][H][W] and t_all[n_samples][c_L][H][W].  losses (host,
 * n_steps doubles, may be NULL) receives each step's loss before its update.
 * Synchronises the stream. */
stg_status stg_cnn_train(stg_cnn* net, const float* x_all, const float* t_all, int n_samples, const int* order,
                         int batch, int n_steps, float lr, double* losses);
/* Text of the last error of this network (NULL net: of the last failed create). */
const char* stg_cnn_last_error(const stg_cnn* net);
stg_status stg_cnn_destroy(stg_cnn* net);

/* Warm-start data of a 2D slab problem (finest level of ctx; STG_EINVAL in 3D).
 * Slab vectors X_* are DEVICE arrays in C-ABI order; v_n = velocity of slab n at its
 * last Radau node (t_n), dv = v_n - v_{n-1}, c_a = Radau nodes on [0, 1].  The image
 * has height = 2 n_y + 1 and width = 2 n_x + 1 (the Q2 nodes, x fastest).
 *   stg_warm_features: feat[2d][H][W] = [v_n / scale_v, dv / scale_d] (components in order).
 *   stg_warm_target:   target[d(k+1)][H][W], channel a*d + comp =
 *                      (v_{n+1}(t_n + c_a tau) - v_n - c_a dv) / scale_d.
 *   stg_warm_start:    X0 (device, N doubles): velocity at node a = v_n + c_a dv
 *                      + scale_d * network(feat)[a*d + comp] (net NULL: the network term
 *                      is left out; it is also left out at Q2 nodes on Dirichlet faces,
 *                      whose data is fixed), pressure at node a = p_n + c_a (p_n - p_{n-1});
 *                      the network must have 2d input and d(k+1) output channels on
 *                      the H x W grid.  Synchronises both streams when net is given.
 *   stg_warm_scales:   root mean squares of the entries of v_n and of dv (host outputs,
 *                      each may be NULL); synchronises. */
stg_status stg_warm_features(stg_ctx* ctx, const double* X_n, const double* X_prev, float scale_v, float scale_d,
                             float* feat);
stg_status stg_warm_target(stg_ctx* ctx, const double* X_n, const double* X_prev, const double* X_next,
                           float scale_d, float* target);
stg_status stg_warm_start(stg_ctx* ctx, stg_cnn* net, const double* X_n, const double* X_prev, float scale_v,
                          float scale_d, double* X0);
stg_status stg_warm_scales(stg_ctx* ctx, const double* X_n, const double* X_prev, double* rms_v, double* rms_dv);

/* Text of the last error of this context (or of the last failed stg_setup
 * when ctx is NULL).  Valid until the next call on the same context. */
const char* stg_last_error(const stg_ctx* ctx);

/* Frees all device memory and the context.  NULL is accepted. */
void stg_destroy(stg_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* STG_H */
