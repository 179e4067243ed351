/*
 * magpie.h -- C ABI of the GB300 (sm_103a) MAGPIE sweep library.
 *
 * MAGPIE (Multilevel-Adaptive-Guided Ptychographic Iterative Engine) solves
 *     min_z  Phi(z) = 1/2 sum_k || Q . P_k z - R_k(P_k z) ||^2      (Eq. exit_misfit)
 * for an object z (n_rows x n_cols, complex) from N diffraction patterns
 * d_k = |F(Q . P_k z*)|^2 (Section 2.1), with a known probe Q (m x m,
 * complex) and scan windows P_k (m x m sub-arrays of z whose top-left corner
 * is positions[k] = (row, col)).  F is the unnormalised 2-D DFT,
 * (Fx)[p,q] = sum_{a,b} x[a,b] exp(-2 pi i (pa + qb)/m), F^{-1} = F^* / m^2.
 *
 * One sweep visits the windows in a caller-supplied permutation (Algorithm
 * MAGPIE), in consecutive minibatches of B windows.  For every window of a
 * minibatch, from the same z: the exit wave Q . z_k, its FFT, the Fourier
 * modulus projection onto sqrt(d_k), the inverse FFT (the revised exit wave
 * R_k of Definition "Revised Exit Wave", with theta(0) := 0), and the MAGPS
 * V-cycle of Algorithm MAGPS with the weights of Eq. (def_weights) and the
 * rPIE regulariser u = alpha (max|Q|^2 - |Q|^2) (Section 2.1).  The
 * increments Delta_k are combined as
 *     z <- z + sum_k P_k^T (w . Delta_k) / sum_k P_k^T w,   w = u + |Q|^2,
 * on pixels where the denominator is positive; for one level this is the
 * exact minimiser of the proximal surrogate of Eq. (proximal_point_method)
 * summed over the minibatch, and for B = 1 it is Algorithm MAGPIE itself.
 *
 * Data types and layouts (all row-major, no padding):
 *   complex   : two float32, real then imaginary (C99 float _Complex,
 *               cuComplex, torch.complex64)
 *   object    : complex [n_rows][n_cols]
 *   probe     : complex [m][m]
 *   positions : int32 [n_pos][2] = (row, col) of the window's top-left pixel,
 *               0 <= row <= n_rows - m, 0 <= col <= n_cols - m
 *   intensities : float32 [n_pos][m][m], DFT order (zero frequency at [0][0],
 *               no FFT shift), non-negative
 *   order / idx : int32 permutation of, or subset of, 0 .. n_pos-1
 *
 * Streams: every call is ordered on the CUDA stream given at creation (a
 * cudaStream_t passed as void*, 0 = the legacy default stream) and returns
 * without waiting for the GPU, except where stated ("synchronous").
 *
 * Errors: every int-returning call returns MAGPIE_OK (0) or a negative code;
 * magpie_strerror() names a code and magpie_last_error() gives the message of
 * the calling thread's most recent failure.  No C++ exception crosses the
 * ABI.  A failed call leaves the context usable unless it returned
 * MAGPIE_ECUDA, after which only magpie_destroy() is meaningful.
 */
#ifndef MAGPIE_H
#define MAGPIE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MAGPIE_OK 0
#define MAGPIE_EINVAL (-1)      /* an argument is out of range or NULL          */
#define MAGPIE_ECUDA (-2)       /* a CUDA runtime call or kernel launch failed  */
#define MAGPIE_ENOMEM (-3)      /* device memory allocation failed              */
#define MAGPIE_EUNSUPPORTED (-4)/* a valid size this build has no kernel for    */
#define MAGPIE_EINDEX (-5)      /* a device-side window index was out of range  */
#define MAGPIE_ETIMEOUT (-6)    /* a bounded device wait ran out (a tcgen05
                                   convolution or transform stopped waiting for
                                   its MMAs, a persistent group step for its
                                   windows, or a precision-form kernel for the
                                   windows handed on by the kernel before it)    */

typedef struct magpie_ctx magpie_ctx;

typedef struct {
  int32_t n_rows, n_cols; /* object size; both >= m                               */
  int32_t m;              /* probe / window side: 8, 16, 32, 64, 128 or 256        */
  int32_t n_pos;          /* N >= 1                                                 */
  int32_t levels;         /* grids including the finest, 1 <= levels <= log2(m)+1;
                             1 is rPIE, L is MAGPIE_{L-1} of Section 5.1            */
  int32_t minibatch;      /* B, 1 <= B <= min(n_pos, 4096)                          */
  float alpha;            /* rPIE constant, finite and >= 0 (Section 2.1)           */
  int32_t update_probe;   /* 0: the probe is known and fixed (the paper); 1: every
                             minibatch step also moves the context's probe (below)  */
  float beta;             /* probe regulariser when update_probe = 1, >= 0          */
  int32_t deterministic;  /* 1: the ordered update (below), bitwise reproducible;
                             0: float-atomic update, the same sums in a run-to-run
                             varying order (last-bit differences)                   */
} magpie_params;

/*
 * The two updates (deterministic = 1 or 0) compute the same combination
 * z <- z + sum_k P_k^T (w . Delta_k) / sum_k P_k^T w of a minibatch:
 *   1  every window writes w . Delta_k to its slot of a minibatch buffer
 *      (8 B m^2 bytes) and an update kernel sums, per object pixel, the
 *      windows covering it in minibatch order: the results are bitwise
 *      reproducible;
 *   0  every window adds (w . Delta_k, w) pixel by pixel into object-sized
 *      accumulators (16 n_rows n_cols bytes) with 16-byte float atomics, and a
 *      streaming kernel applies N / D and clears them: faster, but the
 *      order of the floating-point sums varies from run to run.
 * The atomic update serves the FP32 window kernel (with or without the probe
 * step); the precision form, the learned correction, the phase rule of
 * Eq. (specification) and context groups always use the ordered update.
 */

/*
 * Probe step (update_probe = 1; an extension: the paper keeps Q fixed and
 * names blind ptychography as future work).  From the same (z, Q) as the
 * object step, the surrogate 1/2 || Q . z_k - R_k ||^2, symmetric in Q and
 * z_k, is minimised over Q with a proximal term:
 *   Q <- Q + sum_k conj(z_k)(R_k - Q z_k) / sum_k (u_Q,k + |z_k|^2),
 *   u_Q,k = beta (max |z_k|^2 - |z_k|^2),
 * on probe pixels with a positive denominator; the regulariser and the
 * per-level factors are then recomputed from the new probe.  The context
 * keeps its own probe; magpie_get_probe copies it out.
 */

/*
 * Create a reconstruction context (Algorithm MAGPIE's inputs z^(0), Q,
 * {d_k}, u).  All pointers are DEVICE pointers owned by the caller.
 *   object      : complex [n_rows][n_cols], read and updated in place by the
 *                 sweep calls; must stay allocated while the context lives.
 *   probe       : complex [m][m]; copied at creation (and by
 *                 magpie_set_probe), not kept.
 *   positions   : int32 [n_pos][2]; copied and range-checked at creation
 *                 (this copies them to the host once: synchronous).
 *   intensities : float32 [n_pos][m][m]; read once at creation, when the
 *                 context stores the amplitudes sqrt(d_k) in its own buffer.
 *   stream      : cudaStream_t (as void*) on which every call is ordered.
 * The context owns its workspaces: amplitudes (4 N m^2 bytes), the per-level
 * probe factors, the minibatch increment buffer (8 B m^2 bytes), with
 * deterministic = 0 the object-sized accumulators (16 n_rows n_cols bytes),
 * and small per-window arrays.  Returns MAGPIE_EINVAL for bad sizes, NULL
 * pointers, out-of-range positions or a deterministic value other than 0 or
 * 1, MAGPIE_EUNSUPPORTED for an m without a kernel.
 */
int magpie_create(magpie_ctx** out, const magpie_params* params, void* object,
                  const void* probe, const int32_t* positions,
                  const float* intensities, void* stream);

/* Release every resource of the context (after finishing its stream work). */
void magpie_destroy(magpie_ctx* ctx);

/*
 * One minibatch step of Algorithm MAGPIE (every window of the minibatch from
 * the same object, the combination rule at the top of this file): the windows
 * idx[0..count-1] (DEVICE int32 array) are processed from the current object
 * and their increments applied.  1 <= count <= minibatch.
 * Indices outside [0, n_pos) are skipped on the device and reported as
 * MAGPIE_EINDEX by the next synchronous call.
 */
int magpie_step(magpie_ctx* ctx, const int32_t* idx, int32_t count);

/*
 * One sweep (one iteration of Algorithm MAGPIE): ceil(N / B) minibatch steps
 * over consecutive slices of order[0..n_pos-1] (DEVICE int32 permutation),
 * the last slice possibly shorter.  The order is copied to the context
 * first, so the caller may reuse its buffer once the stream reaches the
 * call.  The steps replay a CUDA graph captured on the first call.
 */
int magpie_sweep(magpie_ctx* ctx, const int32_t* order);

/*
 * One sweep exactly as magpie_sweep, for measurement: the same kernels are
 * launched one by one (not from the graph) with a CUDA event recorded on the
 * context's stream before and after each of them.  Synchronous:
 * writes the summed durations of the per-window kernel (*window_ms) and of the
 * object-update kernel (*apply_ms) over the sweep, and the number of
 * minibatch steps (*launches, one launch of each kernel per step), to HOST
 * pointers (each may be NULL).
 */
int magpie_profile_sweep(magpie_ctx* ctx, const int32_t* order, double* window_ms, double* apply_ms,
                         int32_t* launches);

/* Copy the context's current probe to `probe` (DEVICE complex [m][m]); it
   differs from the one given only with the probe step (an extension). */
int magpie_get_probe(magpie_ctx* ctx, void* probe);

/*
 * Phi(z) of Eq. (exit_misfit) at the current object over all N windows,
 * accumulated in float64 (per window in float32 partial sums of at most a few
 * dozen terms).  Synchronous: writes *phi (HOST pointer).
 */
int magpie_objective(magpie_ctx* ctx, double* phi);

/*
 * The stopping criterion of Section 5, (1/(N m)) sum_k || grad Phi_k(z_k) ||_2
 * with grad Phi_k = conj(Q)(Q z_k - R_k(z_k)) (Eq. misfit_derivative), at
 * the current object over all N windows.  Synchronous: writes *value (HOST).
 */
int magpie_stop_metric(magpie_ctx* ctx, double* value);

/*
 * Re-read the probe from `probe` (DEVICE complex [m][m]) and recompute the
 * regulariser and the per-level factors (Eq. def_weights); `probe` may be
 * the pointer given at creation after the caller changed its contents.
 */
int magpie_set_probe(magpie_ctx* ctx, const void* probe);

/*
 * Per-window values of the last pass over each window (from a sweep, a
 * step or an objective/stop-metric evaluation): phi_k = Phi_k(z_k) (Eq.
 * exit_misfit) and gnorm_k = || grad Phi_k(z_k) ||_2 (Eq. misfit_derivative)
 * at the object the window saw.
 * Synchronous: writes HOST arrays phi[n_pos] and gnorm[n_pos] (either may
 * be NULL).
 */
int magpie_window_values(magpie_ctx* ctx, double* phi, double* gnorm);

/*
 * End-to-end sweep from host memory: copies order (HOST int32[n_pos]) and,
 * if `intensities` (HOST float32 [n_pos][m][m]) is not NULL, a new data set
 * to the device, runs one sweep, and if `object_out` (HOST complex
 * [n_rows][n_cols]) is not NULL copies the object back.  Synchronous.  Host
 * buffers should be page-locked for full copy bandwidth.
 */
int magpie_sweep_host(magpie_ctx* ctx, const int32_t* order, const float* intensities,
                      void* object_out);

/*
 * Pipelined end-to-end sweep from host memory: enqueues, without waiting,
 * the copy of `intensities` (HOST float32 [n_pos][m][m], page-locked for
 * asynchronous copies) and of `order` (HOST int32 [n_pos]) to the device, one
 * sweep on them, and the copy of the object to `object_out` (HOST complex
 * [n_rows][n_cols], may be NULL).  Consecutive calls alternate between two
 * device buffers for the data, and the data copy of a call runs on a copy
 * stream while the previous call's sweep computes, so a sequence of sweeps
 * runs at close to the device rate with every sweep's data brought in anew.
 * The permutation and the data travel on the copy streams; for the FP32 FFT
 * path the window kernels read the raw intensities and take their square
 * roots themselves; an object_out in pinned (mapped) memory is written by a
 * kernel over the host link, other memory by a copy.  Results are those of
 * magpie_sweep_host; the context's own data set and permutation (used by
 * magpie_sweep / magpie_step) are left unchanged.  Host buffers must stay
 * valid and unmodified until magpie_sync returns; magpie_sync waits for all
 * enqueued work and reports errors.
 */
int magpie_sweep_host_async(magpie_ctx* ctx, const int32_t* order, const float* intensities, void* object_out);
int magpie_sync(magpie_ctx* ctx);

/*
 * Forward model of Section 2.1 without noise, d_k = |F(Q . P_k z)|^2 for
 * k = 0..n_pos-1, no context needed.  DEVICE pointers: object complex
 * [n_rows][n_cols], probe complex [m][m], positions int32 [n_pos][2],
 * out float32 [n_pos][m][m].  Same size limits and checks as magpie_create
 * (positions are copied to the host for the range check: synchronous).
 */
int magpie_forward_intensities(const void* object, int32_t n_rows, int32_t n_cols,
                               const void* probe, int32_t m, const int32_t* positions,
                               int32_t n_pos, float* out, void* stream);

/*
 * Context groups: several independent reconstructions advanced together.
 * magpie_group_sweep is one sweep of every member, exactly as magpie_sweep
 * on each of them (member results are bitwise those of separate sweeps), but
 * batched: batched step t runs step t of every member that has one, all
 * windows of equal m in one launch and all members' object updates in one
 * more (or, in the persistent form below, one launch per m for windows and
 * updates together), replayed from one CUDA graph.  Members may differ in
 * every size.
 *   ctxs   : n contexts created on the current device, none with
 *            update_probe = 1, each at most once; they must outlive the group
 *            and not be used on another stream while a group sweep runs.
 *   stream : cudaStream_t (as void*) on which group sweeps are ordered.
 */
typedef struct magpie_group magpie_group;
int magpie_group_create(magpie_group** out, magpie_ctx* const* ctxs, int32_t n, void* stream);

/* orders: HOST array of n DEVICE pointers, orders[i] an int32 permutation of
   0 .. n_pos(i)-1; copied to the members before the sweep. */
int magpie_group_sweep(magpie_group* group, const int32_t* const* orders);

/* Release the group (not its members). */
void magpie_group_destroy(magpie_group* group);

/*
 * The group's autotuner.  magpie_group_create times, for every window side m
 * present in the first batched step, the batched window kernel under each of
 * its candidate register bounds (blocks per SM: the default, an alternative
 * and a denser third: 2 / 1 / 3 for 256-thread blocks, 1 / 2 / 4 for smaller
 * ones, 1 only for m = 256) on that step's own windows, and uses the fastest
 * in every group sweep.  magpie_group_tuning reports, for m = 8, 16, .., 256
 * (index i, m = 8 << i), the bound in use (minb[i]) and the measured ms per
 * launch of the three candidates (ms[3i], ms[3i+1], ms[3i+2]; 0 where not
 * measured or equal to an earlier candidate; HOST arrays of 6 and 18).
 * magpie_group_set_minb forces a candidate.
 */
int magpie_group_tuning(magpie_group* group, int32_t* minb, float* ms);
int magpie_group_set_minb(magpie_group* group, int32_t m, int32_t minb);

/*
 * The autotuner's second dimension: the tile shape of the group's update
 * kernel, one of 16 x 16, 32 x 8 and 32 x 32 pixels per 256-thread block (one,
 * one and four pixels per thread).  magpie_group_create times each on the
 * first batched step with the members' objects replaced by scratch copies
 * (the members' objects are not touched) and uses the fastest.  Every shape
 * sums each pixel's windows in minibatch order, so the results are bitwise
 * identical.  magpie_group_apply_tuning reports the shape in use (*shape, an
 * index 0..2), the three shapes (tile_w[3], tile_h[3]) and their measured ms
 * per launch (ms[3]); HOST pointers.  magpie_group_set_apply_shape forces
 * one (MAGPIE_EINVAL outside 0..2).
 */
int magpie_group_apply_tuning(magpie_group* group, int32_t* shape, int32_t* tile_w, int32_t* tile_h, float* ms);
int magpie_group_set_apply_shape(magpie_group* group, int32_t shape);

/*
 * The autotuner's third dimension: the form of a batched step.
 *   0: separate launches, as above (the batched window kernel per window
 *      side, then one update kernel for all members);
 *   1: persistent, one launch per window side whose clusters (as many as fit
 *      on the GPU at once) take work items from a device queue: first every
 *      window of the side's members, then the members' update tiles (32 x 32
 *      pixels; 16 x 16 for sides below 64).  An update tile waits until every
 *      block of its member's windows has counted itself done, so one member's
 *      update overlaps the other members' windows; the launches of different
 *      sides run concurrently (forked streams in the sweep's graph).  Each wait
 *      is bounded (1 s of GPU time by default): a wait that runs out sets an
 *      error flag and skips its tile, the launch still ends, and
 *      magpie_group_status reports MAGPIE_ETIMEOUT.
 * Both forms sum each pixel's windows in minibatch order and give bitwise
 * identical objects.  magpie_group_create times batched step 0 in both forms
 * (updates writing scratch copies of the objects) and uses the faster.
 * magpie_group_form_tuning reports the form in use (*persistent) and the two
 * measured ms per batched step 0 (ms[2], HOST); magpie_group_set_persistent
 * forces one (MAGPIE_EINVAL unless 0 or 1).  magpie_group_set_wait_limit sets
 * the bound of each wait (seconds in [1e-6, 60]).
 */
int magpie_group_form_tuning(magpie_group* group, int32_t* persistent, float* ms);
int magpie_group_set_persistent(magpie_group* group, int32_t persistent);
int magpie_group_set_wait_limit(magpie_group* group, double seconds);

/* Waits for the group's stream, then reads and clears the error flag of the
   persistent form: MAGPIE_ETIMEOUT if a dependency wait ran out since the
   last call (that update tile was skipped), else MAGPIE_OK. */
int magpie_group_status(magpie_group* group);

/* Self-test of the bounded waits (no counterpart in the paper): runs batched
   step 0 in the persistent form with every update tile waiting for one block
   more than its member's windows have, which never arrives, under a limit of
   `seconds` (in [1e-6, 10]).  Every wait runs out, every update tile is
   skipped (the members' objects are unchanged; their per-window scratch is
   overwritten), the launch ends, and the call returns MAGPIE_ETIMEOUT; the
   group stays usable. */
int magpie_group_check_waits(magpie_group* group, double seconds);

/*
 * Learned coarse-level correction.  The paper has no network: its Algorithm
 * MAGPS ends the recursion on the coarsest grid (side h = m / 2^(levels-1))
 * with one proximal step e_plain = g_H / w_H, g_H = conj(Q_H)(R_H - Q_H z_H)
 * the coarse residual gradient and w_H = u_H + |Q_H|^2.  A context with a
 * network attached lets the network propose that correction instead:
 *   input  x [h][h][4] = (Re z_H, Im z_H, Re e_plain / s, Im e_plain / s),
 *          z_H = the coarse object of the restriction chain
 *          z^{l+1} = I_h^H(W_z^l . z^l) (Eq. def_weights), s = RMS of e_plain
 *          over the window;
 *   output y [h][h][2]; proposal e_nn = e_plain + s (y_re + i y_im).
 * Each window keeps the V-cycle output built on e_nn only when its quadratic
 * surrogate 1/2 ||Q . x - R_k(z_k)||^2 (Eq. quadratic_surrogate) is no larger
 * there than at the output built on e_plain; otherwise the plain output is
 * used.  Everything else in the step is unchanged.
 *
 * The network: six 3x3 convolutions with zero padding (channels 4-32-64-128-
 * 512-64-2; strides 1,2,2,2,1,1; nearest upsampling of the input by 1,1,1,1,
 * 2,4; ReLU after the first five), BF16 weights and activations, FP32
 * accumulation and biases; 980,002 parameters, stored as FP32 in layer order,
 * each layer as weights [c_out][3][3][c_in] then biases [c_out].  All data
 * are NHWC float32 on the DEVICE.
 */
typedef struct magpie_cnn magpie_cnn;

/* Number of parameters (980,002). */
int32_t magpie_cnn_param_count(void);

/* A network for coarsest side h (8, 16, 32 or 64) and batches of at most
   max_batch windows; parameters start at zero.  Calls on it are ordered on
   `stream`. */
int magpie_cnn_create(magpie_cnn** out, int32_t h, int32_t max_batch, void* stream);
/* Frees the network and its buffers (after its stream work); it must not be
   attached to a context that still sweeps. */
void magpie_cnn_destroy(magpie_cnn* cnn);

/*
 * Which kernels the network's forward convolutions use: 1 (the default)
 * the 5th-generation tensor cores (tcgen05.mma, operands in shared memory in
 * the 128-byte-swizzled K-major layout, FP32 accumulators in tensor memory)
 * for every layer whose input and output channels are multiples of 64, and a
 * direct FP32 fused-multiply-add kernel for the thin first (4 -> 32) and last
 * (64 -> 2) layers; 0 the register-fragment mma.sync kernel for every layer.
 * All accumulate the same BF16 products in FP32 (summation order differs).
 * MAGPIE_EINVAL for another value.
 */
int magpie_cnn_set_tensor_path(magpie_cnn* net, int32_t path);

/*
 * Synchronous status of the network's stream: MAGPIE_ETIMEOUT (and the flag
 * cleared) when a tensor-core convolution's bounded wait for its MMAs ran out
 * since the last call (that block skipped its output), else MAGPIE_OK.
 */
int magpie_cnn_status(magpie_cnn* net);

/* Copy in (DEVICE float32 [param_count]) the parameters; resets the Adam
   moments and step count.  magpie_cnn_get_params copies them out. */
int magpie_cnn_set_params(magpie_cnn* cnn, const float* theta);
int magpie_cnn_get_params(magpie_cnn* cnn, float* theta);

/* y [batch][h][h][2] = network(x [batch][h][h][4]); keeps the activations for
   magpie_cnn_backward. */
int magpie_cnn_forward(magpie_cnn* cnn, const float* x, int32_t batch, float* y);

/* grad [param_count] = d<dy, y>/d theta for the inputs of the last forward
   pass (the BF16 roundings passed straight through). */
int magpie_cnn_backward(magpie_cnn* cnn, const float* dy, float* grad);

/*
 * One training step on `batch` trajectories: forward, loss
 * L = 1/2 mean((y - t)^2) with target t = (zh - z_H^0) / s - e_plain / s
 * (x0 = the trajectory's first network input, zh [batch][h][h][2] = its coarse
 * object T V-cycles later, scale [batch] = s), backward, and one Adam step
 * (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) at learning rate lr.
 * loss: DEVICE float64, written when the step runs (no synchronisation).
 */
int magpie_cnn_train_step(magpie_cnn* cnn, const float* x0, const float* zh, const float* scale, int32_t batch,
                          float lr, double* loss);

/* The network input x [count][h][h][4] and s [count] of windows idx[count]
   (count <= minibatch) at the current object; needs levels >= 2, m <= 128 and
   update_probe = 0.  Synchronous (index errors are reported here). */
int magpie_coarse_state(magpie_ctx* ctx, const int32_t* idx, int32_t count, float* x, float* scale);

/* patches [count][m][m] complex = the object's windows idx[count] (zeros for
   an index out of range). */
int magpie_gather_windows(magpie_ctx* ctx, const int32_t* idx, int32_t count, void* patches);

/* Attach a network (NULL detaches): later steps and sweeps of ctx use the
   learned coarse correction.  The network must have h = m / 2^(levels-1) and
   max_batch >= minibatch, must outlive the attachment, and its parameters may
   change between sweeps.  One network serves contexts on one stream. */
int magpie_attach_cnn(magpie_ctx* ctx, magpie_cnn* cnn);

/* Running totals since the first attachment: windows whose proposal was
   evaluated, and windows that kept it.  Synchronous. */
int magpie_learned_stats(magpie_ctx* ctx, int64_t* proposed, int64_t* accepted);

/* For window slots 0..count-1 of the most recent learned step: 1 if the
   learned output was kept, and surrogate(plain) - surrogate(learned).  HOST
   outputs; synchronous. */
int magpie_learned_window_values(magpie_ctx* ctx, int32_t count, int32_t* accepted, double* margin);

/*
 * Precision form: the windows' 2-D DFTs as tensor-core GEMMs.  An m-point
 * line DFT (m = 16 Qr) is two complex matrix products, 16-point DFTs then
 * Qr-point DFTs with FP32 twiddles between them (Cooley-Tukey); each product
 * runs on FP16 tensor cores with hi+lo split operands (a = hi + lo, both
 * FP16, 22 significant bits together; a b taken as hi hi + hi lo + lo hi) and
 * FP32 accumulation.  Each block scales its lines by a power of two into
 * FP16's range and divides the outputs by it (both exact), so any finite
 * input is transformed; a transform carries a relative error of about 5e-7
 * to 7e-7 (the FP32 FFT path about 1e-7).  The projection, the V-cycle and
 * the update are the FP32 path's; Phi_k and the gradient norms stay FP64.
 * mode 0: FP32 FFT path (default); mode 1: tensor-core DFTs with
 * register-fragment MMAs (mma.sync m16n8k16); mode 2: the same DFTs on the
 * 5th-generation tensor cores (tcgen05.mma, operands in shared memory,
 * accumulators in tensor memory; each block's waits on its MMAs are
 * bounded, and one that runs out makes the next objective, stop metric or
 * window-value call return MAGPIE_ETIMEOUT).  Modes 1 and 2 need m = 64, 128
 * or 256 and update_probe = 0.  The mode applies to later steps and sweeps.
 */
int magpie_set_precision(magpie_ctx* ctx, int32_t mode);

/*
 * The transform kernels of a precision-form step hand windows to one another
 * one by one: each kernel lets the next one launch once all of its own
 * blocks run, and a block of the next kernel waits only for the tiles of its
 * own window (a count per window, released by the producer and polled with
 * acquire loads), so that the last wave of one kernel overlaps the first
 * windows of the next.  Every such wait is bounded (0.2 s); one that runs out
 * skips its tile and makes the next objective, stop metric or window-value
 * call return MAGPIE_ETIMEOUT.
 * Self-test of those bounds (no counterpart in the paper): runs the
 * transform and coarse kernels of one step over windows 0 .. min(minibatch,
 * n_pos) - 1 with every wait asking for one tile more than its window has,
 * under a limit of `seconds` (in [1e-6, 10]), and no update.  Every wait
 * runs out, the kernels end, and the call returns MAGPIE_ETIMEOUT; the
 * object is unchanged (the per-window scratch is overwritten) and the
 * context stays usable.  MAGPIE_EINVAL when the context is not in the
 * precision form (mode 1 or 2).  Synchronous.
 */
int magpie_precision_check_waits(magpie_ctx* ctx, double seconds);

/* out[c] = the 2-D DFT of in[c] (unnormalised; inverse = 1: the conjugate
   transform, without 1/m^2) for `count` m x m complex windows (DEVICE), by
   the precision form's tensor-core path: magpie_dft2_tc with mma.sync,
   magpie_dft2_tcgen05 with tcgen05 (MAGPIE_ETIMEOUT if a bounded wait ran
   out).  in == out is allowed.  Allocates a few KiB of tables per call;
   synchronous. */
int magpie_dft2_tc(const void* in, void* out, int32_t m, int32_t count, int32_t inverse, void* stream);
int magpie_dft2_tcgen05(const void* in, void* out, int32_t m, int32_t count, int32_t inverse, void* stream);

/*
 * Variants from the paper, off by default (flags = 0), for later steps and
 * sweeps of ctx:
 *   bit 0  the MG/OPT correction term (Algorithm MG/OPT): every coarse
 *          problem of the V-cycle is the paper's coarse surrogate minus
 *          Re<v_H, z_H>, v_H = grad f_H(z_H) - I_h^H grad f_h(z_h), so the
 *          coarse residual gradient is the plain restriction of the fine one
 *          (needs update_probe = 0).
 *   bit 1  the phase rule of Eq. (specification): where a window's spectrum
 *          entry is exactly 0, the phase of that entry at the window's
 *          previous visit is used (0 on the first visit after this call;
 *          setting the bit again restarts the history).  Keeps one complex
 *          value per window pixel (8 n_pos m^2 bytes).
 * Contexts with bit 1 set cannot join a group.
 */
int magpie_set_variant(magpie_ctx* ctx, int32_t flags);

/* Static name of an error code; never NULL. */
const char* magpie_strerror(int code);

/*
 * One minibatch step, as magpie_step, for callers that cannot allocate GPU
 * memory: code that runs under a fixed memory budget handed out by a host
 * framework, plug-ins whose host application owns every device allocation,
 * and real-time acquisition loops where cudaMalloc's implicit device
 * synchronisation (and its chance of failing under memory pressure) is not
 * acceptable.  It needs no context and calls no allocation routine: its
 * workspace (the per-window increments, the per-level probe factors and the
 * twiddles) lives in one fixed array of about 9.5 MiB that every GPU loading
 * this library holds until the process exits.  This entry point is an
 * addition of this library; the paper has no counterpart.
 *   object      : DEVICE complex [n_rows][n_cols], updated in place
 *   probe       : DEVICE complex [m][m]; its per-level factors are
 *                 recomputed on every call
 *   positions   : DEVICE int32 [n_pos][2]
 *   amplitudes  : DEVICE float32 [n_pos][m][m], the square roots sqrt(d_k)
 *                 of the measured intensities (DFT order)
 *   idx         : DEVICE int32 [count], the windows of this minibatch
 *   phi, gnorm  : DEVICE float64 [n_pos] outputs, Phi_k and ||grad Phi_k||
 *                 of the windows of this minibatch (other entries untouched)
 *   stream      : cudaStream_t as void*
 * Limits: m <= 128 (MAGPIE_EUNSUPPORTED otherwise); 1 <= count <=
 * min(n_pos, 4096) and count * m^2 <= 2^20 (e.g. 64 windows of 128 x 128),
 * otherwise MAGPIE_EINVAL.  Windows whose index or position is
 * out of range are skipped and reported as MAGPIE_EINDEX.  Synchronous: it
 * waits for the step to finish before returning.  The first call on each
 * device looks up the workspace's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  All
 * calls share the one workspace: calls that overlap on the GPU (other
 * threads, other streams) race and must be serialised by the caller.
 */
int magpie_step_noalloc(void* object, int32_t n_rows, int32_t n_cols, const void* probe, int32_t m,
                        const int32_t* positions, int32_t n_pos, const float* amplitudes, const int32_t* idx,
                        int32_t count, int32_t levels, float alpha, double* phi, double* gnorm, void* stream);

/*
 * Thread blocks (one thread-block cluster) per window of the window kernel
 * for window side m, the second dimension of magpie_stage_times' output;
 * 0 for an m without a kernel.
 */
int32_t magpie_window_blocks(int32_t m);

/*
 * Measurement helper, not part of the method: the FP32 fused multiply-add
 * rate of the current device, the peak that bounds the ALU-bound window
 * kernel.  Launches 8 blocks of 256 threads per SM, each thread running 8
 * independent chains of `iters` FMAs, four times on `stream` (the first as a
 * warm-up) and reports the fastest timed launch as *tflops (2 flops per FMA)
 * and *ms (HOST pointers; ms may be NULL).  Allocates a small output buffer;
 * changes no device setting.  Synchronous.
 */
int magpie_fp32_fma_rate(int32_t iters, double* tflops, double* ms, void* stream);

/*
 * Measurement helper, not part of the method: one minibatch step of the FP32
 * form (as magpie_step, object updated) with thread 0 of every block of the
 * window kernel recording %globaltimer (ns) at ten points: start, exit wave
 * gathered, column FFTs sent, row data received, row pass sent, column data
 * received, inverse column FFTs done, g^0 done, block sums done, V-cycle
 * done (0 where a point is not reached).  stamps: HOST uint64
 * [count][blocks per window][10], capacity its length.  Synchronous.
 * Returns MAGPIE_EUNSUPPORTED unless the library was built with
 * MAGPIE_STAGE_TIMES defined (the stamps are compiled out otherwise).
 */
int magpie_stage_times(magpie_ctx* ctx, const int32_t* idx, int32_t count, uint64_t* stamps, int64_t capacity);

/* Message of the calling thread's most recent failed call ("" if none). */
const char* magpie_last_error(void);

/* Library version as major*10000 + minor*100 + patch (this is 1.3.0). */
int magpie_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MAGPIE_H */
