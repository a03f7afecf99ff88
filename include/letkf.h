/*
 * letkf.h - C ABI of libletkf.so, a GB300 (sm_103a) implementation of the
 * per-frame local ensemble transform Kalman filter (LETKF) analysis for
 * adaptive optics, after Gray et al., "Local ensemble transform Kalman filter,
 * a fast non-stationary control law for adaptive optics on ELTs"
 * (arXiv:1408.7069).
 *
 * Model (Section 2.2): the state of actuator node g is the pair
 * (phi_k(g), phi_{k-1}(g)); slopes y_k = D1 phi_{k-1} + w_k with D1 the Fried
 * slope operator (Appendix B) and w_k ~ N(0, sigma2 I); the forecast is the
 * AR(1) model x_{k+1} = A1 x_k + v_k with A1 = [[a I, 0], [I, 0]]
 * (Section 2.2, Eq. Mem_pre).
 *
 * Conventions shared by every entry point:
 *  - Nodes ("points") are the corners of valid subapertures, ordered row-major
 *    over the (nsub+1) x (nsub+1) grid. n_pts of them.
 *  - The ensemble is stored [n_pts][2][m]: row 0 = phi_k, row 1 = phi_{k-1},
 *    member index fastest.
 *  - Slopes y are [p] with p = 2 * (number of valid subapertures): all x-slopes
 *    sx(s,t) = (phi[s+1,t] + phi[s+1,t+1] - phi[s,t] - phi[s,t+1]) / 2 of the
 *    valid subapertures in row-major order, then all y-slopes sy(s,t) =
 *    (phi[s,t+1] + phi[s+1,t+1] - phi[s,t] - phi[s+1,t]) / 2. Radians per
 *    subaperture.
 *  - Floating-point buffers have the handle's storage type: float when
 *    precision = 0, double when precision = 1 ("real" below).
 *  - Pointers named *_dev are device pointers the caller owns; they must stay
 *    valid until the stream reaches the work that uses them. Pointers named
 *    *_host are host pointers read before the call returns.
 *  - Every call is ordered on the handle's CUDA stream and returns without
 *    synchronising, except letkf_create, letkf_destroy, letkf_sync and the
 *    query functions. Faults found on the device (non-finite data, a Jacobi
 *    sweep limit reached) are recorded in a device status word and returned by
 *    the next letkf_sync.
 *  - No C++ exception crosses this boundary; a failing call returns a status and
 *    letkf_last_error() describes it.
 *  - A handle holds one or more independent AO instances (letkf_create_batch).
 *    Per-node, per-slope and per-member buffers of a call are then the
 *    instances' buffers concatenated in instance order: the ensemble is each
 *    instance's [n_pts_i][2][m_i] block in turn, slopes y are p_1 + ... + p_n
 *    values, mean / spread have n_pts_1 + ... + n_pts_n rows of 2, truth has
 *    n_pts_1 + ... values, forecast noise has the [n_pts_i][m_i] blocks in turn,
 *    and a residual call writes one double per instance.
 */
#ifndef LETKF_H
#define LETKF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct letkf_ctx *letkf_t; /* opaque handle owned by the library */

typedef enum {
  LETKF_OK = 0,
  LETKF_ERR_ARG = 1,        /* invalid argument: nothing was launched */
  LETKF_ERR_CUDA = 2,       /* a CUDA runtime call failed */
  LETKF_ERR_NOCONVERGE = 3, /* a Jacobi eigensolve hit its sweep limit */
  LETKF_ERR_TIMEOUT = 4,    /* a bounded device wait gave up */
  LETKF_ERR_NONFINITE = 5,  /* NaN or Inf met in slopes or ensemble */
  LETKF_ERR_STATE = 6,      /* call not valid in the handle's current state */
  LETKF_ERR_NOMEM = 7       /* device or host allocation failed */
} letkf_status;

typedef struct {
  int32_t nsub;                /* subapertures per side; nodes (nsub+1)^2. 1..1024 */
  const uint8_t *subap_mask;   /* host [nsub*nsub] row-major, nonzero = valid; copied */
  int32_t m;                   /* ensemble size, 2..64 (2..32 when precision = 1) */
  int32_t window;              /* localization window: w x w subapertures, odd or even, 1..31 */
  int32_t taper;               /* 0 = box (tau = 1), 1 = Gaspari-Cohn tau on R^-1 */
  double loc_len;              /* Gaspari-Cohn half-support c in pitches; <= 0 -> w / 4 */
  double rho;                  /* multiplicative inflation, > 0 */
  double sigma2;               /* slope noise variance (rad^2), > 0 */
  double a_ar1;                /* AR(1) coefficient of the forecast */
  double noise_std;            /* forecast noise = noise_std * bank screen value */
  int32_t precision;           /* 0 = FP32 storage and analysis with FP64 fallback, 1 = FP64 */
  double fp64_kappa;           /* FP64 fallback threshold on kappa_hat (e.g. 300); <= 0 disables it */
  uint64_t seed;               /* SplitMix64 seed of the forecast-noise draws */
  const float *noise_bank;     /* host [bank_B][bank_G][bank_G] screens, or NULL; copied */
  int32_t bank_B, bank_G;      /* bank shape (ignored when noise_bank is NULL) */
  int32_t max_sweeps;          /* Jacobi sweep limit per node; <= 0 -> 20 */
  int32_t partition;           /* 0: every node is its own local domain (the per-node analysis);
                                  P in 2..64: multi-actuator local domains of a P x P partition
                                  of the node grid (Section 4.1), single instance, FP32, m 2..128;
                                  1: one domain, the global ETKF (Section 3.1.1), m 2..1024 */
  int32_t piston;              /* with partition > 0: nonzero = remove the differential pistons
                                  between domains by least squares (Section 4.4) */
} letkf_config;

/* Validate the configuration, build the node list, the per-node observation
 * windows (Section 4.1: subapertures s in [i - w/2, i - w/2 + w - 1], same
 * for t; Gaspari-Cohn weight of the distance from the node to the subaperture
 * centre), upload masks, windows and the noise bank, and allocate the ensemble
 * (zero: X_{1/0} = 0, Section 3.1) and device scratch. stream: a cudaStream_t
 * (NULL = legacy default stream) on the current device. On success *out owns
 * all of it. */
letkf_status letkf_create(const letkf_config *cfg, void *stream, letkf_t *out);

/* One handle for n independent instances of possibly different sizes (grid,
 * mask, m, window, noise, seeds; one precision for all), analysed together:
 * every frame's kernels cover all instances, analysis tiles of all instances
 * are ordered by cost (largest windows and ensembles first), and letkf_run
 * captures the whole multi-instance frame in one CUDA graph. cfgs: host
 * array of n configurations (masks and banks copied). */
letkf_status letkf_create_batch(const letkf_config *cfgs, int32_t n, void *stream, letkf_t *out);

/* Synchronise the handle's stream and free everything it owns. NULL is a no-op. */
letkf_status letkf_destroy(letkf_t h);

/* Sizes summed over the instances: nodes and slopes; m is the ensemble size of
 * a single-instance handle and 0 for a batch. Host pointers, any may be NULL. */
letkf_status letkf_query(letkf_t h, int32_t *n_pts, int32_t *p, int32_t *m);

/* Sizes of instance i and the number of instances. Host pointers, any may be NULL. */
letkf_status letkf_query_instance(letkf_t h, int32_t i, int32_t *n_pts, int32_t *p, int32_t *m,
                                  int32_t *n_inst);

/* Local domains of a handle created with partition = P > 0 (Section 4.1): the
 * node grid's side of N = nsub + 1 nodes is cut into blocks [floor(b N / P),
 * floor((b + 1) N / P)), b = 0 .. P-1, and the valid nodes of each of the P x P
 * blocks form a domain (empty blocks are dropped; domains are numbered
 * row-major over the blocks). Every domain is analysed as one local problem
 * (Section 4.2) with n_d = 2 x its nodes state rows, observing the union of
 * its nodes' windows with tau = Gaspari-Cohn of the distance from the
 * subaperture centre to the domain's node box (tau = 1 inside it), and with
 * piston != 0 the analysis mean increments are made continuous across domain
 * borders by one least-squares constant per domain and state row (Section 4.4;
 * the constants of each connected group of domains have zero node-weighted
 * mean). letkf_stats then counts in fp64_points the domains whose kappa_hat
 * exceeds fp64_kappa (there is no FP64 path for domains).
 * n_dom: number of domains (0 for a per-node handle); node_dom_host: host
 * int32 [n_pts], the domain of every node; obs_count_host: host int32
 * [n_dom], the number of slopes each domain observes (p_d). Any may be NULL. */
letkf_status letkf_query_domains(letkf_t h, int32_t *n_dom, int32_t *node_dom_host,
                                 int32_t *obs_count_host);

/* Host copies of the node coordinates [n_pts][2] (i, j) and of the number of
 * valid window slopes per node [n_pts] (p_l, Section 4.2's p_d). Either may be NULL. */
letkf_status letkf_query_points(letkf_t h, int32_t *ij_host, int32_t *window_slopes_host);

/* Copy the ensemble [n_pts][2][m] (real) from / into device memory.
 * letkf_set_state also resets every node's stored eigenbasis (the FP32 basis
 * that an analysis hands to its FP64 sweeps and to the reverse mode) to the
 * identity; every analysis writes the bases it reads, so the results that
 * follow depend on the new ensemble only. */
letkf_status letkf_get_state(letkf_t h, void *X_dev);
letkf_status letkf_set_state(letkf_t h, const void *X_dev);

/* Forecast, Section 3.1.2 Eq. Mem_pre with the AR(1) A1 of Section 2.2:
 * phi_{k+1}^i = a phi_k^i + v^i, phi_k^i moved to row 1. noise_dev: device
 * [n_pts][m] real added as v, or NULL to draw v from the noise bank: member i
 * of forecast number f takes screen h % B at offset ((h >> 16) % G,
 * (h >> 40) % G), wrapped, with h = SplitMix64(seed, f * 2^16 + i), times
 * noise_std. Increments the handle's forecast counter f. */
letkf_status letkf_forecast(letkf_t h, const void *noise_dev);

/* Local analysis of every node (Section 4.2 with Section 3.1 and Appendix A):
 * mean and anomalies of the background, slope anomalies Yb = D1 (phi_{k-1}
 * anomalies), innovations d = y - D1 mean(phi_{k-1}); per node, with the
 * window's slopes and R_l^-1 = diag(tau_j / sigma2): A = (m-1)/rho I + C Yb_l,
 * C = Yb_l^T R_l^-1, A = Q Lambda Q^T, wbar = Q Lambda^-1 Q^T C d,
 * W = Q ((m-1) Lambda^-1)^(1/2) Q^T, X_a = xbar + X_b' (wbar 1^T + W).
 * y_dev: device [p] real. mean_dev, spread_dev: device [n_pts][2] real or
 * NULL; spread is the sample standard deviation over members (m - 1). The
 * ensemble is replaced by the analysis.
 * FP32 handles: a node whose kappa_hat = 1 + rho tr(C Yb_l) / (m - 1), an upper
 * bound on the condition number of A, exceeds fp64_kappa is analysed in FP64
 * (Gram and accumulated Jacobi sweep, started from the node's FP32 eigenbasis)
 * and written back in FP32. */
letkf_status letkf_analyze(letkf_t h, const void *y_dev, void *mean_dev, void *spread_dev);

/* Loop criterion (Section 2.1 Eq. Crit_Opt; Section 5): spatial variance over
 * nodes of truth - mean(row 0), piston removed, of the current (forecast)
 * ensemble. truth_dev: device [n_pts] real. resvar_dev: device double[1]. */
letkf_status letkf_residual(letkf_t h, const void *truth_dev, double *resvar_dev);

/* Closed loop over `frames` frames: for frame k, the residual of the current
 * prediction against truth_seq[k] into resvar[k], the analysis of
 * y_seq[k], then a forecast with bank noise. y_seq_dev: device [frames][p]
 * real; truth_seq_dev: device [frames][n_pts] real or NULL (then no residual);
 * resvar_dev: device double[frames][n_inst] or NULL. use_graph != 0 captures
 * one frame of every instance into a CUDA graph once and replays it. Requires a
 * noise bank for every instance. */
letkf_status letkf_run(letkf_t h, int32_t frames, const void *y_seq_dev, const void *truth_seq_dev,
                       double *resvar_dev, int32_t use_graph);

/* The closed loop of letkf_run over `frames` frames (1..65536) as ONE launch:
 * every frame of every instance (residual, observation, analysis, forecast)
 * is captured into one CUDA graph, instantiated once per (frames, pointers)
 * and launched once, so the host takes no part between frames. Same results
 * as letkf_run, bit for bit. stamps_dev: device uint64_t[frames + 1] or NULL;
 * element 0 receives the global timer (ns) at the start of the launch and
 * element k + 1 once frame k has completed, so per-frame times are taken
 * inside the launch. Requires a non-default stream and a noise bank for every
 * instance. */
letkf_status letkf_run_graph(letkf_t h, int32_t frames, const void *y_seq_dev,
                             const void *truth_seq_dev, double *resvar_dev, uint64_t *stamps_dev);

/* Deformable mirror of a single-instance per-node handle (Section 2.1, Eqs.
 * Eq_Obs and Eq_Cor; Section 2.2; Appendix B.3): n = n_pts; N is the influence
 * matrix (row b, column a: the phase at node b per unit command of actuator
 * a; actuators at the nodes) and P the command matrix (the least-squares
 * projection (N^T N)^-1 N^T of Appendix B.3, as the caller calibrated it),
 * both host CSR: int32 row pointers [n + 1], int32 column indices, double
 * values; copied (to the handle's real type). The library forms D1 N (at
 * most 36 nonzeros per row for a 5 x 5 influence support) and zeroes the
 * commands. From then on
 *  - letkf_analyze takes y as the measurement of the residual phase, y_k =
 *    D1 (phi^tur_{k-1} - N u_{k-2}) + w_k, and analyses the pseudo-open-loop
 *    slopes y_k + D1 N u_{k-2} (ybar of Section 3.1.1 with its D1 N term);
 *  - every forecast is followed by the command u_k = P phihat_{k+1/k}, the
 *    predicted turbulent phase (row 0 mean) projected on the mirror;
 *  - letkf_residual measures phi^tur_k - N u_{k-1}, the residual phase left
 *    by the applied correction;
 * the commands live on the device in a ring of three indexed by the forecast
 * counter (so frames stay graph-capturable; letkf_set_frame moves it too).
 * n_ptr NULL removes the mirror (the pseudo-open-loop form: the correction
 * is the prediction itself). LETKF_ERR_ARG for a batch or domain handle or
 * malformed CSR. Synchronises. */
letkf_status letkf_set_dm(letkf_t h, int32_t n, const int32_t *n_ptr, const int32_t *n_idx,
                          const double *n_val, const int32_t *p_ptr, const int32_t *p_idx,
                          const double *p_val);

/* The latest command u (the one computed after the last forecast), device
 * [n_pts] real: what a controller sends to the mirror. Stream-ordered. */
letkf_status letkf_get_command(letkf_t h, void *u_dev);

/* The simulated true closed loop with the handle's deformable mirror over
 * `frames` frames: for frame k the residual variance of phi^tur_k - N u_{k-1}
 * into resvar[k] (if not NULL), the measurement y_k = D1 (phi^tur_{k-1} -
 * N u_{k-2}) + w_k (phi^tur_{k-1} = truth_seq[k - 1], zero for the call's first
 * frame), the analysis, the forecast with bank noise and the command.
 * truth_seq_dev: device [frames][n_pts] real; wnoise_seq_dev: device
 * [frames][p] real (w_k); resvar_dev: device double[frames] or NULL.
 * use_graph != 0 replays one captured frame. LETKF_ERR_STATE without a mirror
 * or a noise bank. */
letkf_status letkf_run_dm(letkf_t h, int32_t frames, const void *truth_seq_dev,
                          const void *wnoise_seq_dev, double *resvar_dev, int32_t use_graph);

/* Change instance i's inflation rho, slope noise variance sigma2 and taper
 * half-support loc_len (<= 0: window / 4) in place (Section 4.2: A = (m-1)/rho I
 * + Yb^T R^-1 Yb with R^-1 = diag(tau_j / sigma2)); the next analysis uses them.
 * LETKF_ERR_ARG unless rho, sigma2 > 0 and all are finite. Synchronises. */
letkf_status letkf_set_params(letkf_t h, int32_t i, double rho, double sigma2, double loc_len);

/* Stopping rule of the FP32 Jacobi eigensolve (Section 4.2's EVD, one-sided
 * Jacobi on A's columns). A column pair is rotated when the cosine of its
 * angle exceeds rotate_tol (default 4e-6); a node's solve stops after a sweep
 * in which every rotated pair had a cosine of at most stop_cos (default 1e-3;
 * values below rotate_tol mean rotate_tol, i.e. stop after a sweep without
 * rotations). Measured at the ELT steady state against the FP64 oracle,
 * teacher-forced: the default gives 2e-6 on the analysis mean, 1e-5 on the
 * spread and 4e-5 on the anomalies with 5.7 sweeps per node; stop_cos =
 * rotate_tol gives 2e-6 / 3e-6 / 9e-6 with 8.3 sweeps. FP64 handles and the
 * FP64 fallback keep their own tolerance. LETKF_ERR_ARG outside (0, 1) and
 * [0, 1). Synchronises. */
letkf_status letkf_set_jacobi(letkf_t h, double rotate_tol, double stop_cos);

/* Set the forecast counter: the next forecast with bank noise draws the noise
 * of frame `frame` (>= 0) and later ones follow on. A new handle starts at 0.
 * Synchronises. */
letkf_status letkf_set_frame(letkf_t h, int64_t frame);

/* One closed-loop frame from host memory, for a real-time controller: copies
 * y_host [p] (real) and, if not NULL, truth_host [n_pts] into pinned staging
 * buffers the handle owns, runs the frame as letkf_run does (residual of the
 * current prediction against truth, analysis of y, forecast with bank noise),
 * waits for it, and copies the analysis mean [n_pts][2] (real) into mean_host
 * and the residual variance (one double per instance) into resvar_host (either
 * may be NULL; resvar_host only with truth_host). The frame runs as one CUDA
 * graph (captured on the first call, per with/without truth) on a non-default
 * stream. Requires a noise bank for every instance. It returns once the
 * outputs are in host memory; the frame's forecast may still be running on
 * the handle's stream then, and every later call on the handle is ordered
 * after it. On the legacy default stream it synchronises the stream. */
letkf_status letkf_step(letkf_t h, const void *y_host, const void *truth_host, void *mean_host,
                        double *resvar_host);

/* Reverse mode of the closed loop. J = mean over `frames` frames of the
 * residual variance of the prediction (Section 2.1 Eq. Crit_Opt, as in
 * letkf_residual), each frame run as in letkf_run (residual of the current
 * prediction, analysis of y_seq[k] by Section 4.2, forecast of Section 3.1.2
 * with bank noise) from the handle's current ensemble, eigenbases and frame
 * counter; and grad = (dJ/drho, dJ/dsigma2, dJ/dL), L the Gaspari-Cohn
 * half-support of the taper (cfg.loc_len, or window / 4 when that is <= 0; the
 * L component is 0 without the taper). The analysis is differentiated through
 * its eigendecomposition with divided differences of lambda^-1/2 written in a
 * form exact for equal eigenvalues, so windows with fewer slopes than m - 1
 * (exactly degenerate eigenvalues) need no special case. The backward pass
 * recomputes each node's eigenbasis from the one its forward analysis stored
 * (FP32), and in FP64 for the nodes that the FP64 fallback takes.
 * y_seq_dev: device [frames][p] real; truth_seq_dev: device [frames][n_pts] real.
 * ckpt_every: frames per segment; the forward keeps the ensemble and bases at
 *   the start of every segment and the backward recomputes one segment at a
 *   time (device memory ~ (frames / ckpt_every + ckpt_every) states); <= 0 or
 *   >= frames keeps every frame (no recomputation).
 * J_out, grad_out: host double[1] and double[3], either may be NULL.
 * Single-instance handles with m <= 32 and a noise bank only (LETKF_ERR_ARG /
 * LETKF_ERR_STATE otherwise). On return the handle holds the state letkf_run
 * would leave after the same frames. With a non-default stream the whole
 * computation is captured once into a CUDA graph (rebuilt when the sequence
 * pointers, frames or ckpt_every change) and replayed. Synchronises. The
 * result is bitwise reproducible for the same inputs. */
letkf_status letkf_grad(letkf_t h, int32_t frames, const void *y_seq_dev, const void *truth_seq_dev,
                        int32_t ckpt_every, double *J_out, double *grad_out);

/* Analysis tile shapes. On FP32 handles the analysis runs one CTA per tile of
 * tile_i x tile_j nodes (4, 2 or 1 nodes per warp for m <= 16, <= 32 and
 * larger) and stages the tile's window halo in shared memory once (FP64
 * handles run one CTA of four warps per node and ignore the shapes); the best shape depends on the window, the ensemble size and the
 * mix of instances. letkf_tile_shape describes compiled shape number `shape`
 * (0 .. count-1; LETKF_ERR_ARG beyond). Instances are grouped in width classes
 * by ensemble size: 0 for m <= 16, 1 for m <= 32, 2 for m <= 64 (one node per
 * warp, tiles of at most 8 nodes). On FP32 handles a tile
 * holds whole warps of nodes (a multiple of 4 nodes in class 0, of 2 in class
 * 1); a shape a class cannot take gives LETKF_ERR_ARG. New handles start at
 * shape 0 (2 x 4). letkf_set_tile_shape
 * selects a shape for one class; letkf_autotune times every allowed shape for every class
 * present on the handle's current ensemble with slopes y_dev (reps timed
 * analyses of that class's nodes each, state restored afterwards; tune on a
 * loop state, not on a fresh prior draw whose nodes mostly take the FP64
 * path), keeps the fastest and writes the
 * choices to shapes_out[3] and their analysis time in microseconds to us_out[3]
 * (either may be NULL; on FP64 handles it times nothing, returns the current
 * shapes and zero times). Both synchronise; choices may be cached by the caller
 * and restored with letkf_set_tile_shape. */
letkf_status letkf_tile_shape(int32_t shape, int32_t *tile_i, int32_t *tile_j);
letkf_status letkf_set_tile_shape(letkf_t h, int32_t width_class, int32_t shape);
letkf_status letkf_autotune(letkf_t h, const void *y_dev, int32_t reps, int32_t *shapes_out,
                            float *us_out);

/* Row split of the FP32 per-node analysis (Section 4.2's eigensolve and
 * transform), per width class: split = 1 (the default) gives each lane two
 * whole columns of the node's matrix; split = 2 gives each lane the rows of
 * one half of two columns, so a node takes twice the lanes (2 nodes per warp
 * for m <= 16, 1 for m <= 32), every dot product of the one-sided Jacobi adds
 * its partner lane's half, and a rotation round's dependent chain is about
 * half as long. It pays on systems whose nodes fill few warps per SM (a few
 * thousand nodes or fewer on 152 SMs) and costs issue slots on large ones.
 * The results differ from split 1 by rounding only (sums in another order);
 * for fixed settings they are bitwise reproducible. Width classes 0 and 1 of
 * FP32 per-node handles only, with the class's current tile shape holding
 * whole warps of nodes in the split form; LETKF_ERR_ARG otherwise (FP64 and
 * domain handles, class 2, split not 1 or 2). Synchronises; drops the cached
 * CUDA graphs. letkf_autotune keeps the split and times the shapes it allows. */
letkf_status letkf_set_row_split(letkf_t h, int32_t width_class, int32_t split);

/* Start of the FP64 eigensolve on FP64 handles (Section 4.2's EVD): warm = 1
 * (the default) runs the FP32 two-columns-per-lane eigensolve on the window
 * rounded to FP32 first and starts each node's FP64 one-sided Jacobi from that
 * basis, made orthonormal to FP64 rounding by two Newton-Schulz steps, stopping after a
 * sweep whose cosines all stay below 1e-8 (the next would rotate by about its
 * square); warm = 0 starts from the identity and stops after a sweep without
 * rotations. Both give FP64 results (they differ by rounding). FP64 per-node
 * handles only (LETKF_ERR_ARG otherwise). The FP32 pass takes the class's
 * tile shape, so FP64 handles take the shapes of the whole-column FP32 form.
 * Synchronises; drops the cached CUDA graphs. */
letkf_status letkf_set_fp64_start(letkf_t h, int32_t warm);

/* Synchronise the stream, return and clear the first error recorded on the
 * device since the last call (LETKF_OK if none). */
letkf_status letkf_sync(letkf_t h);

/* Counters of the last analysis, host pointers (any may be NULL): nodes that
 * took the FP64 fallback, the largest and the total number of Jacobi sweeps
 * over the nodes (a node of the FP64 fallback counts the sweeps of its FP32
 * and of its FP64 eigensolve). Synchronises. */
letkf_status letkf_stats(letkf_t h, int32_t *fp64_points, int32_t *max_sweeps,
                         int32_t *total_sweeps);

/* Allocation-free analysis of one frame, for callers that cannot allocate
 * device memory once running (a real-time controller whose memory is fixed at
 * start-up, or code where cudaMalloc is not allowed). It needs no handle and
 * calls no cudaMalloc, cudaFree or other allocating routine: its scratch (the
 * slope-anomaly and innovation grids, node tables, counters) is one static
 * device array of about 6 MB that every GPU loading this library keeps until
 * the process exits. The paper has no counterpart; it computes the same
 * analysis as letkf_analyze in FP32, with eigenvectors accumulated from the
 * identity and without the FP64 fallback.
 * cfg: as for letkf_create (host mask read during the call); precision must be
 *   0 and nsub <= 128, m <= 32, window <= 15, otherwise LETKF_ERR_ARG with the
 *   limits in errbuf. Noise-bank fields are ignored.
 * X_dev: device float [n_pts][2][m], background in, analysis out.
 * y_dev: device float [p]. mean_dev, spread_dev: device float [n_pts][2] or NULL.
 * stream: cudaStream_t for all of the work (NULL = legacy default stream).
 * errbuf: caller buffer of errlen bytes for a message on failure, or NULL.
 * cfg->fp64_kappa > 0: nodes whose kappa_hat (see letkf_analyze) exceeds it
 *   are counted (this path has no FP64 fallback: their mean may miss the FP32
 *   tolerance); letkf_noalloc_status reports the count.
 * The first call on a device looks up the array's device address. The call
 * copies its tables from host memory that the next call reuses, so it cannot
 * be captured into a CUDA graph: on a capturing stream it returns
 * LETKF_ERR_ARG and launches nothing. Every call shares the array and
 * overwrites its contents (the grids and the status counters are cleared at
 * the start of each call); calls whose GPU work overlaps (other streams, other
 * host threads) race. Faults found on the device are not returned by this
 * call: read them with letkf_noalloc_status. */
letkf_status letkf_analyze_noalloc(const letkf_config *cfg, void *X_dev, const void *y_dev,
                                   void *mean_dev, void *spread_dev, void *stream, char *errbuf,
                                   size_t errlen);

/* Status of the last letkf_analyze_noalloc call on the current device, for the
 * same callers (it allocates nothing either). Synchronises `stream` (the
 * stream of that call), then reads the status word from the static array:
 * LETKF_ERR_NONFINITE if a node met NaN or Inf, else LETKF_ERR_NOCONVERGE if a
 * node reached the sweep limit, else LETKF_OK; LETKF_ERR_CUDA if a CUDA call
 * failed. kappa_nodes (host, may be NULL): the number of nodes whose kappa_hat
 * exceeded cfg->fp64_kappa in that call. The paper has no counterpart. */
letkf_status letkf_noalloc_status(void *stream, int32_t *kappa_nodes);

/* Measured arithmetic peaks of the current device, the denominators of the
 * analysis roofline (the analysis is bound by FP32 arithmetic, its fallback by
 * FP64). Independent FMA chains in every thread of a grid of 4 CTAs of 256
 * threads per SM, timed with CUDA events after a warm-up launch; the SM clock
 * is read from clock64 and the global timer of every CTA. out: host double[7]:
 * FP32 TFLOP/s with scalar FMAs and the SM MHz during that kernel, FP32 TFLOP/s
 * with packed two-wide FMAs and its MHz, FP64 TFLOP/s and its MHz, the SM
 * count (an FMA counts as two flops). Takes about 0.1 s; allocates and frees
 * device memory; synchronises. It changes no clock or other device setting.
 * The paper has no counterpart. */
letkf_status letkf_fma_peaks(double *out);

/* Where the FP32 analysis kernel spends its time, in a library built with
 * phase clocks (build option LK_PHASE_CLOCKS; LETKF_ERR_STATE otherwise):
 * SM cycles summed over its warps since the last call, out: host uint64_t[5]
 * = halo staging, Gram and kappa_hat, Jacobi sweeps, eigenpairs + transform +
 * apply (Section 4.2's steps), and the number of warps. Synchronises the
 * device and resets the counts. The paper has no counterpart. */
letkf_status letkf_phase_clocks(uint64_t *out);

/* The same for the reverse mode's node kernel (letkf_grad): SM cycles summed
 * over its nodes since the last call, out: host uint64_t[12], [0..5] for its
 * FP32 form and [6..11] for its FP64 form (FP64 handles and the queued nodes
 * of FP32 handles) = window staging, Gram and the start of the eigensolve
 * (B = A U0, or the FP64 warm basis), Jacobi sweeps, the adjoint of the
 * transform up to A_bar, the window slopes' adjoints, and the number of nodes.
 * LETKF_ERR_STATE without phase clocks. Synchronises the device and resets
 * the counts. */
letkf_status letkf_adjoint_phase_clocks(uint64_t *out);

/* Text of the last error on this handle (or of the last failed create when h is NULL). */
const char *letkf_last_error(letkf_t h);

#ifdef __cplusplus
}
#endif
#endif /* LETKF_H */
