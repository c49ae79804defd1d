/*
 * fewha.h -- C ABI of libfewha.so, the FEWHA hot path on one B300 (sm_103a).
 *
 * FEWHA (Finite Element Wavelet Hybrid Algorithm) solves the discretised MAP
 * normal equations of atmospheric tomography (Sec. 2.2, Eq. (fewha)):
 *
 *     M c = b,  M = W P^T Gamma^T C^{-1} Gamma P W^T + alpha D,
 *               b = W P^T Gamma^T C^{-1} s,
 *
 * by a few iterations of Jacobi-preconditioned CG (Alg. 2), warm-started from
 * the previous frame (Alg. 1), followed by the mirror fit and gain (Alg. 1).
 * W is the periodic orthonormal db3 wavelet transform of each layer, P the
 * bilinear layer-to-sensor propagation (cone effect for laser guide stars,
 * Sec. 2.1), Gamma the Shack-Hartmann operator on the bilinear grid (Sec. 2.1),
 * C^{-1} the diagonal noise weight and D a diagonal wavelet-domain
 * regulariser (Sec. 2.2).
 *
 * Conventions used by every entry point:
 *   - Every function returns an int status: FEWHA_OK or one FEWHA_ERR_* code;
 *     fewha_last_error() gives a message.  No C++ exception crosses the ABI.
 *   - The handle owns all device state.  Input pointers are borrowed for the
 *     duration of the call only (their contents are copied).
 *   - Arrays are in the handle's precision (float for FEWHA_FP32, double for
 *     FEWHA_FP64).  on_device = 1: a device pointer on this GPU, ordered on the
 *     handle's stream; on_device = 0: a host pointer (the call then
 *     synchronises the stream where it must read or write host memory).
 *   - Work is enqueued on the stream given to fewha_create (0 = legacy
 *     default stream); only calls that touch host memory, fewha_sync and
 *     fewha_get_* with host pointers synchronise.
 *   - Layouts (row-major, "y" = row index i, "x" = column index j):
 *       layers / wavelet coefficients: [layer][y][x], layer-major, n_l x n_l
 *         each, Mallat layout for coefficients (Sec. 2.2, Table 1);
 *       slopes: [wfs][x-slopes | y-slopes][i][j], n_sub x n_sub each (Sec. 2.1);
 *       mirror commands: [dm][y][x], n_act x n_act each.
 */
#ifndef FEWHA_H
#define FEWHA_H

#ifdef __cplusplus
extern "C" {
#endif

#define FEWHA_OK            0
#define FEWHA_ERR_ARG       1   /* invalid argument (null, size, range)                 */
#define FEWHA_ERR_INPUT     2   /* non-finite slopes detected on the device             */
#define FEWHA_ERR_GEOMETRY  3   /* a sample point falls outside a layer or mirror grid  */
#define FEWHA_ERR_BREAKDOWN 4   /* PCG step denominator <= 0 or non-finite (Alg. 2)     */
#define FEWHA_ERR_TIMEOUT   5   /* a bounded grid barrier expired; state left unchanged */
#define FEWHA_ERR_LAUNCH    6   /* the persistent kernel cannot be made co-resident     */
#define FEWHA_ERR_CUDA      7   /* a CUDA runtime call failed                           */
#define FEWHA_ERR_STATE     8   /* call out of order (e.g. solve before set_frame)      */

#define FEWHA_FP32 0
#define FEWHA_FP64 1

#define FEWHA_PATH_PLAIN 0      /* one simple kernel per operator (FP32 or FP64)       */
#define FEWHA_PATH_FUSED 1      /* persistent whole-frame kernel (FP32 only)           */

#define FEWHA_MAX_WFS      16
#define FEWHA_MAX_LAYERS   64
#define FEWHA_MAX_DMS      8
#define FEWHA_MAX_FIT_DIRS 64
#define FEWHA_MAX_JACOBI_LEVELS 16

/* Operating modes of the mirror fit (Sec. 1, Sec. 4.3). */
#define FEWHA_FIT_MCAO 0
#define FEWHA_FIT_MOAO 1

/* Telescope, guide stars / wavefront sensors, mirrors, fitting directions.
 * Angles in radians, heights and lengths in metres (Sec. 2.1, Sec. 4.1). */
typedef struct {
    double D;                              /* telescope diameter                                */
    double obstruction;                    /* central obstruction, diameter ratio [0, 1)        */
    int    n_wfs;                          /* number of Shack-Hartmann sensors (1..MAX_WFS)     */
    int    n_sub[FEWHA_MAX_WFS];           /* subapertures per side of each sensor (>= 1)       */
    double theta_x[FEWHA_MAX_WFS];         /* guide-star direction                              */
    double theta_y[FEWHA_MAX_WFS];
    double gs_height[FEWHA_MAX_WFS];       /* LGS height H (cone factor 1 - h/H); 0 = NGS       */
    double noise_sigma[FEWHA_MAX_WFS];     /* slope noise std (rad); C^{-1} = mask / sigma^2    */
    int    n_dm;                           /* deformable mirrors for the fit (0 = no fit)       */
    double dm_height[FEWHA_MAX_DMS];
    double dm_pitch[FEWHA_MAX_DMS];        /* actuator pitch                                    */
    int    n_fit_dir;                      /* fitting directions (NGS-type)                     */
    double fit_theta_x[FEWHA_MAX_FIT_DIRS];
    double fit_theta_y[FEWHA_MAX_FIT_DIRS];
    int    fit_n_sub;                      /* pupil sample grid of the fit: fit_n_sub+1 nodes   */
    int    precision;                      /* FEWHA_FP32 or FEWHA_FP64, fixed at create         */
    int    lgs_tt_filter;                  /* 1: LGS sensors do not sense tip/tilt: their       */
                                           /* C^{-1} removes each slope axis' mean over active  */
                                           /* subapertures (plain path, and the fused path with */
                                           /* the level-stacked layer phase; batches and        */
                                           /* differentiation refuse it)                        */
    int    fit_mode;                       /* FEWHA_FIT_MCAO: every mirror over every fitting   */
                                           /* direction (one mirror, one direction: LTAO);      */
                                           /* FEWHA_FIT_MOAO: mirror t fitted in direction t    */
                                           /* alone (n_dm == n_fit_dir; open loop only)         */
} fewha_geometry;

/* Turbulence layers reconstructed (Sec. 2.1 layered model; Table 1 sizes). */
typedef struct {
    int    n_layers;                       /* 1..MAX_LAYERS                                     */
    double height[FEWHA_MAX_LAYERS];       /* m                                                 */
    double cn2[FEWHA_MAX_LAYERS];          /* Cn^2 fraction gamma_l (> 0), enters D as 1/gamma  */
    int    n_side[FEWHA_MAX_LAYERS];       /* layer grid n_l: power of two, 8..1024             */
    int    levels[FEWHA_MAX_LAYERS];       /* db3 levels J_l, 1 <= J_l, n_l >> J_l >= 2         */
    double r0;                             /* Fried parameter at 500 nm (m)                     */
    double alpha;                          /* regularisation weight alpha (> 0), Eq. (fewha)    */
    double jacobi_level_weight[FEWHA_MAX_JACOBI_LEVELS];
                                           /* modified Jacobi: the preconditioner's diagonal of */
                                           /* a level-j coefficient (j = 1 finest) is          */
                                           /* weight[j-1] * diag(M); 0 (the default) means 1    */
} fewha_profile;

typedef struct fewha_handle fewha_handle;

/* Build all geometry tables (layer grids, sample/gather tables, D, Jacobi
 * J = diag(M)) on the host in FP64, allocate device state (cudaMalloc) on the
 * current device and upload.  The state (c, b, r, mirror commands) starts at
 * zero.  stream: a cudaStream_t (may be 0).  On failure *out is NULL and the
 * message is available from fewha_last_error(NULL).  Errors: ARG, GEOMETRY
 * (a sensor or fitting footprint leaves a layer grid), CUDA. */
int fewha_create(const fewha_geometry* geom, const fewha_profile* prof, void* stream,
                 fewha_handle** out);

/* Free all device and host memory of the handle (synchronises its stream). */
int fewha_destroy(fewha_handle* h);

/* Message of the last error on this handle (h = NULL: of the last failed
 * fewha_create in this thread).  The pointer stays valid until the next call. */
const char* fewha_last_error(const fewha_handle* h);

/* Sizes: N coefficients (sum n_l^2), S slopes (sum 2 n_sub^2), A actuators. */
int fewha_sizes(const fewha_handle* h, long* n_coeff, long* n_slopes, long* n_act);

/* Select the execution path for FP32 handles (FP64 handles always use the
 * plain path).  Default: FEWHA_PATH_FUSED for FP32 when a fused plan exists
 * for the geometry, else FEWHA_PATH_PLAIN.  Requesting FEWHA_PATH_FUSED
 * without a plan returns FEWHA_ERR_GEOMETRY (fewha_last_error says why: too
 * many layers or sensors, shared memory, the LGS tip-tilt filter on a plan
 * that only fits the row-stripe layer phase) and keeps the current path. */
int fewha_set_path(fewha_handle* h, int path);

/* Residual replacement period k_rr (Alg. 1 warm restart, reading: every
 * k_rr-th frame r = b - M c instead of r = (b - b_prev) + r_prev); 0 = never.
 * Default 10. */
int fewha_set_residual_replacement(fewha_handle* h, int k_rr);

/* Copy the measurement vector s (S values, slopes layout above) into the
 * handle (Alg. 1 input s).  Masked subapertures are ignored by the solve. */
int fewha_set_frame(fewha_handle* h, const void* slopes, int on_device);

/* Alg. 1 up to the PCG: b1 = W P^T Gamma^T C^{-1} s; warm_start = 1:
 * r = (b1 - b0) + r0 (or the replacement), c from the previous frame;
 * warm_start = 0: c = 0, r = b1.  Then n_iter iterations of Alg. 2
 * (n_iter >= 1).  Asynchronous; errors detected on the device (INPUT,
 * BREAKDOWN, TIMEOUT) are reported by the next fewha_sync. */
int fewha_solve(fewha_handle* h, int n_iter, int warm_start);

/* Alg. 1 fitting and gain: a~ = F W^{-1} c, then a1 = (1 - gain) a0 + gain a~
 * (open loop) or a1 = a0 + gain (a~ - a^(-1)) (closed loop, fewha_set_loop).
 * F: least squares over the fitting directions, n_fit CG iterations
 * warm-started from the previous a~; or, when there are as many mirrors as
 * layers and mirror m sits at layer m's height (Sec. 4.1, L = M), the
 * sampling of layer m at mirror m's actuators (n_fit is then ignored).
 * dm_out (A values, may be NULL) receives a1.  Errors: STATE if the geometry
 * has no mirrors. */
int fewha_fit_dm(fewha_handle* h, double gain, int n_fit, void* dm_out, int on_device);

/* phi = W^{-1} c (N values, layers layout). */
int fewha_get_layers(fewha_handle* h, void* out, int on_device);

/* Vectors of the solver state, N values each: which = 0 c, 1 r, 2 b,
 * 3 Jacobi diagonal diag(M), 4 alpha*D.  Host copies synchronise. */
int fewha_get_vector(fewha_handle* h, int which, void* out, int on_device);

/* Checkpoint / resume of the Alg. 1 state (c0, b0, r0): N values each. */
int fewha_get_state(fewha_handle* h, void* c, void* b, void* r, int on_device);
int fewha_set_state(fewha_handle* h, const void* c, const void* b, const void* r, int on_device,
                    long frame_count);

/* y = M x (N values each), one operator application (Eq. (fewha) left side). */
int fewha_apply_M(fewha_handle* h, const void* x, void* y, int on_device);

#define FEWHA_OP_W       0
#define FEWHA_OP_WT      1
#define FEWHA_OP_P       2
#define FEWHA_OP_PT      3
#define FEWHA_OP_GAMMA   4
#define FEWHA_OP_GAMMA_T 5

/* The single operators of M (plain kernels, the handle's precision):
 *   FEWHA_OP_W        coefficients = W layers (periodic db3 analysis, Sec. 2.2), N -> N
 *   FEWHA_OP_WT       layers = W^T coefficients (synthesis, W^-1 = W^T),           N -> N
 *   FEWHA_OP_P        sensor nodes = P layers (every sensor, Sec. 2.1),             N -> NW
 *   FEWHA_OP_PT       layers = P^T sensor nodes (deterministic gather),            NW -> N
 *   FEWHA_OP_GAMMA    slopes = Gamma nodes (every subaperture, unweighted),        NW -> S
 *   FEWHA_OP_GAMMA_T  nodes = Gamma^T slopes,                                       S -> NW
 * with NW the sensor nodes, sum (n_sub + 1)^2, layout [sensor][i][j].
 * fewha_operator_dims gives the input and output lengths. */
int fewha_operator_dims(fewha_handle* h, int op, long* n_in, long* n_out);
int fewha_apply_operator(fewha_handle* h, int op, const void* x, void* y, int on_device);

/* Profiling aid: mean duration (us, CUDA events on the handle's stream) of
 * one application of operator op over reps back-to-back applications on the
 * handle's own buffers (after one untimed application).  Synchronises. */
int fewha_time_operator(fewha_handle* h, int op, int reps, double* us_per_application);

/* One whole frame of Alg. 1 as one CUDA graph: copy in the slopes s, RHS,
 * warm restart, n_iter iterations of Alg. 2, optional fit + gain (dm_out),
 * optional layers phi = W^{-1} c (layers_out), copy out.  on_device = 0: the
 * three pointers are host memory (pinned memory is used in place, pageable
 * memory is staged) and the call synchronises; on_device = 1: device
 * pointers, the call only enqueues.  A host frame on the fused path without
 * dm_out returns as soon as the kernel has set the handle's completion word
 * (mapped pinned memory, written after every result is visible to the host):
 * the results and the error status are final then, while the launch may
 * still be retiring on the stream (later calls are ordered after it).  With
 * pinned slopes and layers there (open loop, slopes by copy, the default of
 * fewha_set_host_transfer) the frame runs as an armed frame fired at once
 * (fewha_frame_arm + fewha_frame_fire below): the kernel is launched first
 * and does its set-up while the copy engine brings the slopes in, on a
 * second stream, and lets it go.  Otherwise the graph is captured on the
 * first call and re-captured when n_iter, the flags or the pointers change;
 * frames that fall on the residual-replacement period use a second graph.
 * layers_out / dm_out may be NULL. */
int fewha_frame(fewha_handle* h, const void* slopes, int n_iter, int warm_start,
                double gain, int n_fit, void* layers_out, void* dm_out, int on_device);

/* Profiling aid: host-side timing of the last fewha_frame on this handle, in
 * microseconds of the host's steady clock: out[0] preparation (argument
 * checks, pointer lookups, graph capture or re-pointing), out[1] the graph
 * launch call (the kernel's launch for a frame run as an armed one), out[2]
 * the wait for the results (host frames on the fused
 * path: until the completion word is seen; 0 for device frames), out[3] the
 * whole call; out[4] = 1 if the captured kernel node was re-pointed at other
 * buffers, out[5] = 1 if the graph was (re)captured.  Errors: ARG. */
int fewha_get_frame_timing(fewha_handle* h, double* out);

/* Loop mode of Alg. 1 (default open).  closed = 1: every frame first forms
 * the pseudo-open-loop slopes s + Gamma P_DM a^(-1) -- the measurements the
 * mirror shapes of two frames back add in every sensor: mirror m (height h_m)
 * sampled bilinearly at the sensor's nodes with the shift theta_g h_m and,
 * for a laser guide star, the cone factor 1 - h_m/H_g, then Gamma, added on
 * every subaperture -- and the fit's gain becomes a^(1) = a^(0) + gain
 * (a~ - a^(-1)).  The input slopes are the residual measurements.  Errors:
 * STATE (no mirrors), GEOMETRY (a sensor sees beyond a mirror grid; the
 * mirrors are sized for the fitting directions), ARG. */
int fewha_set_loop(fewha_handle* h, int closed);

/* The paper has no counterpart: how a host frame's slopes reach the fused
 * kernel (fewha_frame with host buffers).  slopes_by_copy = 1 (default): one
 * copy-engine transfer of the pinned slopes into the handle's slope buffer
 * precedes the kernel in the frame's graph; 0: the kernel reads them through
 * the pinned buffer's device mapping.  The layers come back through the
 * mapping either way (posted writes), and the host waits on the completion
 * word.  On a host link where the kernel's reads wait a round trip each,
 * the copy is the faster of the two.  Drops the captured frame graphs.
 * Errors: ARG. */
int fewha_set_host_transfer(fewha_handle* h, int slopes_by_copy);

/* The paper has no counterpart: a host frame armed ahead of its slopes, for a
 * real-time loop (Alg. 1 per frame, as fewha_frame with host buffers and no
 * mirror fit, open loop, fused path).  fewha_frame_arm launches the frame's
 * kernel now; it does its set-up (L2 prefetch, descriptors, first tables)
 * and then waits, at most wait_s seconds (0 < wait_s <= 60), for
 * fewha_frame_fire before it reads the slopes.  The caller fills the slopes
 * array between the two calls (it must stay valid until fire returns);
 * fewha_frame_fire lets the kernel go, waits for the frame's completion word
 * and returns its status, with the layers in layers_out.  slopes / layers_out:
 * pinned host buffers (device-mapped), read and written by the kernel
 * through the mapping.  The launch latency is thereby taken off the path
 * from the slopes' arrival to the layers.  The armed kernel occupies the GPU
 * while it waits; every other call on the handle but fewha_frame_fire,
 * fewha_sync and the queries returns STATE until the frame is fired.
 * Without a fire by the deadline the frame does no work and fire reports
 * TIMEOUT (the state is untouched; the frame counter has advanced: restore
 * it with fewha_set_state if the replacement schedule matters).
 * Errors: ARG (null or unmapped buffers, wait_s), STATE (no fused plan,
 * closed loop, already armed / nothing armed), then the frame's own. */
int fewha_frame_arm(fewha_handle* h, const void* slopes, int n_iter, int warm_start, void* layers_out, double wait_s);
int fewha_frame_fire(fewha_handle* h);

/* Wait for the handle's stream and return the device error word (OK, INPUT,
 * BREAKDOWN, TIMEOUT).  The word is cleared after it has been read. */
int fewha_sync(fewha_handle* h);

/* Grid-barrier spin budget of the fused kernel in clock cycles (0 makes every
 * barrier expire at once; used to exercise the TIMEOUT path).  Default 2^31. */
int fewha_set_barrier_budget(fewha_handle* h, long long cycles);

/* Fused-path shape (FP32 handles): rebuild the plan with thread-block
 * clusters of cluster_size CTAs per layer (1, 2, 4, 8 or 16).  Errors: ARG
 * if no plan of that size fits the geometry or the device. */
int fewha_set_cluster_size(fewha_handle* h, int cluster_size);

/* Fused-path layer phase (FP32 handles): form = 0 keeps each layer in row
 * stripes of its cluster and runs the 2D DWT of Sec. 2.2 level by level (one
 * cluster barrier per level whose block spans CTAs); form = 1 runs it
 * level-stacked: every column of the CTA's column stripe through the whole 1D
 * cascade, one exchange of the stacked rows through distributed shared
 * memory, then a 1D cascade per row (and the transposes in reverse for W^T),
 * the same coefficients in Mallat layout; form = -1 (the default) takes the
 * level-stacked form wherever it fits shared memory.  The plan is rebuilt
 * (with the current cluster size when that size supports the form).
 * Errors: ARG (no plan of that form fits), STATE (FP64 handle). */
int fewha_set_layer_transform(fewha_handle* h, int form);

/* Autotuner of the fused path: times every feasible cluster shape (and, unless
 * fewha_set_layer_transform fixed it, both layer-phase forms) on the
 * current frame (set_frame first) for n_iter warm-started iterations, reps
 * timed launches each (CUDA events, median), keeps the fastest and restores
 * the solver state (c, r, b) it found.  report (len bytes, may be NULL)
 * receives the timings.  Synchronises.  Errors: STATE (FP64 handle or no
 * frame), ARG. */
int fewha_autotune(fewha_handle* h, int n_iter, int reps, char* report, int len);

/* Kernel launches enqueued by this handle since creation (all paths). */
long long fewha_launch_count(const fewha_handle* h);

/* One-line summary of the execution plan (precision, path, sizes; for the
 * fused path the cluster shape, grid, shared memory and work items), written
 * into buf (len bytes, NUL-terminated, truncated if short). */
int fewha_describe(fewha_handle* h, char* buf, int len);

/* Phase trace of the fused kernel (a profiling aid, off by default).  on = 1:
 * every following fused launch records, per CTA, the globaltimer (ns) when it
 * arrives at and leaves each grid barrier (slot 0 = kernel start, the last
 * slot = kernel end).  fewha_get_trace synchronises and copies the last
 * launch's record, laid out [slot][cta][arrive, depart] (at most max_entries
 * values; out may be NULL to query the sizes), and returns the slot and CTA
 * counts.  Errors: STATE on the plain path. */
int fewha_set_trace(fewha_handle* h, int on);
int fewha_get_trace(fewha_handle* h, unsigned long long* out, int max_entries, int* slots, int* grid);

/* Marks inside the phases of the last traced fused launch (profiling aid):
 * per CTA a row of per_cta values (tag << 56 | globaltimer ns), 0 = unused.
 * Tags: 10..16 layer phase (start, sensor rows staged, P^T done, forward DWT
 * done, update done, inverse DWT done, end), 17 / 18 inside the update of an
 * iteration (scalars known, elementwise loop done); 20..24 sensor tile (start,
 * windows staged, P done, slopes done, end); 30 RHS sensor tile start;
 * level-stacked layer phase: 50 column cascade (and its stores into the rows'
 * owners) done, 51 first cluster barrier passed, 53 row synthesis done, 54
 * second cluster barrier passed.
 * Synchronises.  Errors: STATE on the plain path. */
int fewha_get_fine_trace(fewha_handle* h, unsigned long long* out, int max_entries, int* per_cta, int* grid);

/* ------------------------------------------------------------------------
 * Differentiation of the solve (reverse mode).  The reconstruction of Alg. 1
 * is a fixed, small number of Alg. 2 steps, so its output is a smooth
 * function of the model parameters of Sec. 2.2: the Cn^2 fractions gamma_l
 * (through D ~ 1/gamma_l), the regularisation weight alpha and the sensor
 * weights w_g = 1/sigma_g^2 of C^{-1} (in M and in b).  These calls give the
 * gradient of a loss on the layers phi = W^T c_K of a cold-started K-step
 * solve, with the Jacobi preconditioner held fixed (a constant of the
 * differentiated map).  All array arguments are device pointers in the
 * handle's precision (gradients: double) ordered on the handle's stream; the
 * calls only enqueue.  They use the plain operator kernels and do not touch
 * the frame state (c, r, b) of fewha_solve / fewha_frame.
 * ------------------------------------------------------------------------ */

/* Replace gamma_l (n_layers values > 0), alpha (> 0) and w_g (n_wfs values
 * >= 0) for every later call (M, b, the fused and plain paths).  The Jacobi
 * diagonal keeps its create-time value.  Synchronises the stream.
 * Errors: ARG. */
int fewha_set_params(fewha_handle* h, const double* cn2_frac, double alpha, const double* w);

/* Bytes of device memory a taped solve of n_iter iterations records
 * (5 n_iter vectors of N plus 8 n_iter doubles); -1 on bad arguments. */
long fewha_tape_bytes(const fewha_handle* h, int n_iter);

/* Differentiable solve: b from the slopes (Alg. 1), c = 0, r = b, n_iter steps
 * of Alg. 2, every iterate recorded in `tape` (caller-owned device memory of
 * fewha_tape_bytes bytes, 8-byte aligned); layers_out (may be NULL) = W^T c.
 * Errors: ARG; BREAKDOWN / INPUT are reported by fewha_sync. */
int fewha_solve_taped(fewha_handle* h, const void* slopes, int n_iter, void* tape, void* layers_out);

/* Reverse mode of fewha_solve_taped (same slopes, n_iter and tape, and the
 * parameters the tape was recorded with): for the cotangent layers_bar =
 * dLoss/dphi it writes dLoss/dgamma (n_layers doubles), dLoss/dalpha (1) and
 * dLoss/dw (n_wfs) -- overwritten, not accumulated -- and, if grad_slopes is
 * not NULL, dLoss/dslopes = C^{-1} Gamma P W^T b-bar (slope layout).
 * Errors: ARG. */
int fewha_backward(fewha_handle* h, const void* slopes, int n_iter, const void* tape, const void* layers_bar,
                   double* grad_cn2, double* grad_alpha, double* grad_w, void* grad_slopes);

/* Bytes of device memory a taped solve of n_frames frames records together
 * (5 n_iter n_frames vectors of N plus 8 n_iter n_frames doubles); equal to
 * fewha_tape_bytes for one frame; -1 on bad arguments. */
long fewha_tape_bytes_batch(const fewha_handle* h, int n_iter, int n_frames);

/* fewha_solve_taped for n_frames frames at once (1..65535; the autograd batch
 * of a training step): slopes [n_frames][S], layers_out [n_frames][N] (may be
 * NULL), one tape of fewha_tape_bytes_batch bytes holding every frame's
 * iterates.  Each frame is its own cold-started solve with the same
 * operator; every kernel of the chain processes all frames in one launch
 * (the frame is the grid's third axis), so the launch count does not grow
 * with n_frames.  Errors: ARG; BREAKDOWN / INPUT by fewha_sync. */
int fewha_solve_taped_batch(fewha_handle* h, int n_frames, const void* slopes, int n_iter, void* tape,
                            void* layers_out);

/* Reverse mode of fewha_solve_taped_batch (same n_frames, slopes, n_iter,
 * tape and parameters): layers_bar [n_frames][N]; per frame gradients, each
 * overwritten: grad_cn2 [n_frames][n_layers], grad_alpha [n_frames],
 * grad_w [n_frames][n_wfs], and, if not NULL, grad_slopes [n_frames][S].
 * Errors: ARG. */
int fewha_backward_batch(fewha_handle* h, int n_frames, const void* slopes, int n_iter, const void* tape,
                         const void* layers_bar, double* grad_cn2, double* grad_alpha, double* grad_w,
                         void* grad_slopes);

/* ------------------------------------------------------------------------
 * Batch of independent instances.  Sec. 4 finds the global parallelism of a
 * single reconstruction (a handful of layers and sensors) far too small to
 * fill a GPU; a batch advances many unrelated FP32 instances (different
 * telescopes, sensors, layer grids) together, each by the frame of Alg. 1
 * (RHS, warm restart with residual replacement every k_rr frames, n_iter
 * steps of Alg. 2) exactly as fewha_solve does for one handle, in one launch
 * of the persistent fused kernel per frame -- or one launch per group of
 * instances, one after another on the stream, when the batch is split
 * (fewha_batch_set_groups, or the autotuner splitting it by layer size).
 * Instances share nothing but a launch: every one keeps its own tables,
 * state and CG scalars.
 *   slopes: the instances' slope vectors concatenated in instance order
 *           (slope_off[i] .. slope_off[i+1]), each laid out as for a handle;
 *   layers: the instances' layer stacks concatenated (coeff_off[i] ..).
 * ------------------------------------------------------------------------ */
typedef struct fewha_batch fewha_batch;

/* Create a batch of count instances; geoms[i] / profs[i] as for fewha_create
 * (precision must be FEWHA_FP32).  max_tile_side > 0 bounds the sensor tiles
 * (nodes per side) so that large and small sensors give work items of
 * similar size; 0 = one tile per CTA share.  cluster_size 0 = automatic, else
 * 1, 2, 4, 8 or 16 CTAs per layer item.  On failure *out = NULL and
 * fewha_batch_last_error(NULL) gives the reason.  Errors: ARG, GEOMETRY (an
 * instance's geometry, or no fused plan fits the batch), CUDA. */
int fewha_batch_create(int count, const fewha_geometry* geoms, const fewha_profile* profs, void* stream,
                       int max_tile_side, int cluster_size, fewha_batch** out);
int fewha_batch_destroy(fewha_batch* b);
const char* fewha_batch_last_error(const fewha_batch* b);

/* Instance count and total sizes; coeff_off / slope_off (count + 1 entries
 * each, may be NULL) receive the offsets of every instance. */
int fewha_batch_sizes(const fewha_batch* b, int* count, long* coeff_off, long* slope_off);

/* Residual replacement period of the batch (as fewha_set_residual_replacement). */
int fewha_batch_set_residual_replacement(fewha_batch* b, int k_rr);

/* One frame for every instance: copy the slopes in, the fused launches (one
 * per group), copy the layers phi = W^T c out (layers_out may be NULL).  on_device = 0: host
 * buffers, the call synchronises and returns the device error word (INPUT if
 * any instance's slopes are non-finite, BREAKDOWN if any instance's CG step
 * broke down -- that instance keeps its state -- or TIMEOUT). */
int fewha_batch_frame(fewha_batch* b, const void* slopes, int n_iter, int warm_start, void* layers_out,
                      int on_device);

/* State (c, the previous right-hand side b, r) of instance inst, as
 * fewha_get_state.  Synchronises for host pointers. */
int fewha_batch_get_state(fewha_batch* b, int inst, void* c, void* bprev, void* r, int on_device);

/* Wait for the batch's stream and return its device error word (cleared). */
int fewha_batch_sync(fewha_batch* b);
int fewha_batch_describe(fewha_batch* b, char* buf, int len);
long long fewha_batch_launch_count(const fewha_batch* b);

/* Autotuner of the batch's launches.  The instances are grouped by layer
 * size (an instance's largest layer side; a group is a range of the sorted
 * distinct sides: every split between them for up to four sides, at most one
 * split for more); for every group it builds the plan for every cluster size
 * (8, 4, 16, 2) and sensor-tile bound (none, 64, 48, 32, 24, 16) that fits
 * shared memory and times each on the current slopes (n_iter warm-started
 * iterations from the same state, CUDA events, median of reps launches after
 * one warm-up).  A grouping costs the sum of its groups' best launches; the
 * cheapest replaces the current launches if it beats them (timed the same
 * way), and the instances' state is restored.  report: the timings
 * (NUL-terminated, truncated to len).  Synchronises. */
int fewha_batch_autotune(fewha_batch* b, int n_iter, int reps, char* report, int len);

/* Split the batch into launches by hand: group[i] (count = the instance
 * count entries) is the launch of instance i, 0 .. G - 1 with every launch
 * non-empty; launches run in index order, each with its own plan built with
 * the batch's max_tile_side and cluster_size.  The instances keep their
 * state.  Synchronises.  Errors: ARG (a bad or missing index), GEOMETRY (no
 * plan fits a group: the current launches stay), CUDA. */
int fewha_batch_set_groups(fewha_batch* b, const int* group, int count);

/* Bound on the launches per frame that fewha_batch_autotune may choose
 * (0 = none, the default; 1 = the whole batch in one launch).  The current
 * launches are replaced by the autotuner's choice when they exceed the
 * bound.  Errors: ARG (NULL handle or a negative bound). */
int fewha_batch_set_max_launches(fewha_batch* b, int max_launches);

/* Sub-phase marks of a batch's fused launches, as fewha_set_trace /
 * fewha_get_fine_trace for one handle (the same tags; a CTA's marks follow
 * its sensor tiles and layer items in order, up to the per-CTA capacity
 * *per_cta).  fewha_batch_get_fine_trace synchronises and copies the last
 * traced frame's marks: the CTAs of the first launch, then those of the
 * next (*grid counts them all; the timestamps share one clock).  Errors:
 * ARG. */
int fewha_batch_set_trace(fewha_batch* b, int on);
int fewha_batch_get_fine_trace(fewha_batch* b, unsigned long long* out, int max_entries, int* per_cta, int* grid);

/* Profiling aid for the roofline of the fused kernel (Sec. 4.3 places the
 * operators of M against a memory roofline; the fused kernel's working set
 * stays in L2, so the L2, not HBM, is its bandwidth bound): the achievable
 * L2 bandwidth of the current device, measured with the library's own
 * kernels.  A device buffer of `bytes` (a multiple of 256 in 1..96 MiB, well
 * below the 126 MB L2; allocated and freed by the call) is written once, then
 * read -- and copied, its first half into its second -- `passes` times per
 * launch with 16-byte loads and stores that bypass L1; each of the two
 * kernels is timed over `reps` launches (CUDA events on a private stream) and
 * the fastest launch gives read_gbs (bytes read / s) and copy_gbs (bytes read
 * + written / s), in GB/s.  Synchronises.  errbuf (errlen bytes, may be NULL)
 * receives a message on failure.  Errors: ARG (range), CUDA. */
int fewha_measure_l2(long bytes, int passes, int reps, double* read_gbs, double* copy_gbs, char* errbuf,
                     int errlen);

/* The paper has no counterpart: this entry point serves callers that cannot
 * allocate device memory (a control loop that reserves all memory at start-up
 * and allows no allocation while it runs, code inside a framework that owns
 * the device memory).  It computes layers = W^{-1} coeffs, the same layer
 * reconstruction as fewha_get_layers, for a stack of n_layers FP32 layers
 * without a handle and without allocating anything.  coeffs / layers: device
 * pointers, sum n_side[l]^2 floats each, layer-major, Mallat layout in, nodal
 * values out; they must not overlap.  n_side[l]: power of two in 8..1024;
 * levels[l]: 1 <= J, n_side >> J >= 2.  Work is enqueued on `stream`
 * (0 = legacy default stream); the call does not wait for it.
 * The intermediate of each level lives in one fixed 4 MiB array that every
 * GPU loading the library reserves until exit, so the total coefficient count
 * may not exceed 2^20 (ARG error with a message otherwise).  The first call on
 * a device looks up that array's address; make it before any stream capture.
 * Every call reuses the same array: calls that overlap on the GPU race.
 * errbuf (errlen bytes, may be NULL) receives a message on failure.
 * Errors: ARG (null, aliasing or out-of-range sizes), CUDA. */
int fewha_layers_noalloc(const float* coeffs, float* layers, int n_layers, const int* n_side,
                         const int* levels, void* stream, char* errbuf, int errlen);

/* Sites of the debug build's bounds checks (fewha_debug_bounds): the sensor
 * tile's bilinear reads of the layers (WIN_SRC; WIN_DST and WIN_P belonged
 * to the staged windows the tile no longer uses and stay reserved), slope
 * indices and Gamma^T output; the layer phase's field staging source and destination,
 * P^T gather reads, level-stacked DWT stores into row and column owners,
 * coefficient indices, tip-tilt correction nodes, layer output; the
 * row-stripe DWT's peer reads; table staging; the plain path's P, P^T and
 * Gamma / Gamma^T; the fit; the no-allocation transform. */
enum {
    FEWHA_DBG_WIN_SRC = 1, FEWHA_DBG_WIN_DST = 2, FEWHA_DBG_WIN_P = 3, FEWHA_DBG_SLOPES = 4,
    FEWHA_DBG_GT_OUT = 5, FEWHA_DBG_STG_SRC = 6, FEWHA_DBG_STG_DST = 7, FEWHA_DBG_PT_READ = 8,
    FEWHA_DBG_CASC_OWN = 9, FEWHA_DBG_CASC_COL = 10, FEWHA_DBG_COEF = 11, FEWHA_DBG_TT = 12,
    FEWHA_DBG_PHI_OUT = 13, FEWHA_DBG_STRIPE = 14, FEWHA_DBG_TABLES = 15, FEWHA_DBG_PLAIN_P = 16,
    FEWHA_DBG_PLAIN_PT = 17, FEWHA_DBG_PLAIN_GAMMA = 18, FEWHA_DBG_FIT = 19, FEWHA_DBG_NOALLOC = 20
};

/* The paper has no counterpart: the memory checker of the debug build.  A
 * library built with -DFEWHA_DEBUG (libfewha_debug.so, made next to the
 * release library) checks at every gather and scatter of the hot path --
 * the fused kernel's field staging, bilinear reads, P^T gather,
 * DWT exchange stores and coefficient indices; the plain path's P, P^T,
 * Gamma and Gamma^T; the fit's sparse products and layer samples; the
 * no-allocation transform -- that the index lies inside the buffer it
 * addresses, and skips the access where it does not.  This call reports and
 * clears the violations recorded since the last call, over every kernel of
 * the library: *count their number, *first the first one as
 * (site << 48) | (index & (2^48 - 1)), site one of the FEWHA_DBG_* values
 * below.  Synchronises with the device.  Returns 1 in a debug build, 0 in
 * the release build (which checks nothing: both outputs 0), FEWHA_ERR_CUDA
 * if reading the records failed, FEWHA_ERR_ARG for null pointers. */
int fewha_debug_bounds(unsigned long long* first, unsigned long long* count);

#ifdef __cplusplus
}
#endif
#endif /* FEWHA_H */
