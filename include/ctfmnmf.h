/*
 * ctfmnmf.h -- C ABI of libctfmnmf: CTF-MNMF with iterative source steering (ISS)
 * on one NVIDIA GB300 (sm_103a).
 *
 * Method: Xie, Wang, Zhang, Yang, Makino, "Accelerated Convolutive Transfer
 * Function-Based Multichannel NMF Using Iterative Source Steering" (APSIPA ASC 2025).
 *   - extended instantaneous model, rows r <-> (source n, tap l), sum_n L_n = M   (Sec. II, Eq. 3)
 *   - demixing y_{r,i,j} = w_r^H x_{i,j}                                          (Eq. 4)
 *   - NMF source model lambda_{n,i,j} = sum_k T[n,i,k] V[n,k,j]                    (Sec. II)
 *   - negative log-likelihood                                                     (Eq. 5)
 *   - ISS rank-1 updates W_i <- W_i - z_r w_r^H with the closed form of Eq. 16    (Sec. III-A)
 *   - multiplicative updates of T (Eq. 17) and V (Eq. 18), scale normalisation    (Sec. III-A)
 *   - source images by the multichannel Wiener filter                            (Eqs. 23-24)
 *
 * Conventions for every entry point:
 *   - The return value is a ctfmnmf_status: 0 on success, a negative code on failure.
 *     No call aborts, traps or exits the process. After a failure,
 *     ctfmnmf_last_error(h) returns a short static description.
 *   - "device pointer" means memory of the GPU current when the handle was created
 *     (cudaMalloc or a torch CUDA tensor). The caller owns every pointer it passes;
 *     the library never frees or retains caller memory after the call returns.
 *   - "host pointer" means ordinary or pinned CPU memory.
 *   - complex64 = two float32 (re, im), interleaved, as cuFloatComplex / torch.complex64.
 *   - Arrays are dense, C order, with the stated shapes and no padding.
 *   - Dimensions: M microphones, N sources, B NMF bases per source (the paper's K_n),
 *     F frequency bins (the paper's I), J frames, L_n taps of source n with sum L_n = M.
 *   - Work is enqueued on the handle's stream (ctfmnmf_set_stream; default: the legacy
 *     default stream) and is asynchronous unless the entry point says it synchronises.
 *   - A handle is not thread-safe: calls on one handle must be serialised by the caller.
 */
#ifndef CTFMNMF_H
#define CTFMNMF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CTFMNMF_MAX_M 8   /* most microphones (= extended rows) per mixture          */
#define CTFMNMF_MAX_B 32  /* most NMF bases per source                                */

typedef enum ctfmnmf_status {
    CTFMNMF_OK = 0,
    CTFMNMF_EINVAL = -1,       /* bad argument: shape, null pointer, option value          */
    CTFMNMF_ESTATE = -2,       /* call out of order, e.g. iterate before load_stft         */
    CTFMNMF_ECUDA = -3,        /* a CUDA runtime call failed                              */
    CTFMNMF_ENONFINITE = -4,   /* the input STFT or NMF factors hold NaN or Inf          */
    CTFMNMF_ETIMEOUT = -5,     /* a bounded device-side wait gave up                     */
    CTFMNMF_ENOMEM = -6,       /* device allocation failed                                */
    CTFMNMF_EUNSUPPORTED = -7, /* valid shape that these kernels do not handle (see create) */
    CTFMNMF_EBOUNDS = -8       /* a device-side bounds check of a CTFMNMF_DEBUG build stopped
                                  a thread block before an out-of-range access             */
} ctfmnmf_status;

/* Activation update variants (Eq. 18). */
enum {
    CTFMNMF_V_ALL_TAPS = 0,    /* default: sum over all taps of the source, the
                                  majorisation-minimisation form of Eq. 18            */
    CTFMNMF_V_TAP0 = 1         /* Eq. 18 as printed: tap l = 0 only                    */
};

typedef struct ctfmnmf_dims {
    int M, N, L, B, F, J;      /* L: cap on taps per source (and the length of the
                                  mixing CTF the data was made with)                   */
} ctfmnmf_dims;

typedef struct ctfmnmf_options {
    int v_update;              /* CTFMNMF_V_ALL_TAPS (default) or CTFMNMF_V_TAP0        */
    int normalize;             /* 1 (default): scale normalisation of Eqs. 19-21 after
                                  every iteration; 0: none                              */
    int use_graph;             /* 1 (default): the two-kernel path replays a CUDA graph
                                  of its launches; 0: plain stream launches             */
    int path;                  /* CTFMNMF_PATH_AUTO (default), _TWO_KERNEL or _PERSISTENT */
    int wait_timeout_ms;       /* bound of every device-side wait of the persistent path;
                                  0 (default) = 2000 ms. A wait that runs out ends the
                                  launch and the next ctfmnmf_synchronize (or any call that
                                  synchronises) returns CTFMNMF_ETIMEOUT                 */
    int w_update;              /* CTFMNMF_W_ISS (default): the ISS sweep of Eqs. 11-16;
                                  CTFMNMF_W_IP: the IP update of Eqs. 9-10 that ISS
                                  replaces (M <= 4, two-kernel path only, not in a batch;
                                  keeps a copy of X, 8*M*F*J more bytes)                */
    int bin_fpt;               /* frames per thread of the two-kernel bin phase: 1, 2, 4
                                  or 8 (M <= 4) frames strided by the block size when it
                                  fits J; -8: eight consecutive frames per thread in the
                                  kernel compiled for the default taps (M <= 4, taps as
                                  ctfmnmf_create derives them, J <= 4096); 0 (default):
                                  with path AUTO timed among the candidates, else the
                                  fewest that fit. EUNSUPPORTED if the value cannot run
                                  this shape                                              */
    float eps_floor;           /* floor of T and V after each multiplicative update and at
                                  set_init; 0 (default) = 1e-12. Must be >= 0 and finite  */
    int deterministic_reduce;  /* 1 (default): every reduction in a fixed order, so that a
                                  run repeats bit for bit; 0: the long-J cluster bin phase
                                  may add its row powers with shared-memory atomics      */
    int check_finite;          /* 1: scan Y, T and V for NaN/Inf after every iteration of
                                  the two-kernel path (after the whole call on the
                                  persistent path); the next synchronising call returns
                                  CTFMNMF_ENONFINITE and the state must be reloaded.
                                  0 (default): no scan. Builds made with -DCTFMNMF_DEBUG
                                  always scan                                            */
    int reserved[1];           /* must be zero                                          */
} ctfmnmf_options;

/* Demixing updates (ctfmnmf_options.w_update). */
enum {
    CTFMNMF_W_ISS = 0,
    CTFMNMF_W_IP = 1
};

/* Execution paths of ctfmnmf_iterate. PERSISTENT: all iterations of a call in one
 * cooperative launch with a grid-wide barrier between the per-bin and the cross-bin
 * steps (needs B <= 16, J <= 4096 for M <= 4 or J <= 2048 for M = 5..8, and enough
 * co-resident thread blocks). TWO_KERNEL: one launch per step, replayed as a CUDA graph.
 * AUTO: when the persistent path fits, ctfmnmf_create_ex times a few iterations of each path
 * on a probe state and keeps the faster (synchronous, a few milliseconds; the handle then
 * holds the default factors and no STFT, as any new handle); else two-kernel.
 * ctfmnmf_get_path reports the choice. */
enum {
    CTFMNMF_PATH_AUTO = 0,
    CTFMNMF_PATH_TWO_KERNEL = 1,
    CTFMNMF_PATH_PERSISTENT = 2
};

typedef struct ctfmnmf* ctfmnmf_t;

/* Fill *opt with the defaults listed above. */
void ctfmnmf_default_options(ctfmnmf_options* opt);

/*
 * Create a solver for one mixture on the current CUDA device and allocate its
 * device state (about 8*M*F*J + 12*N*F*J + 4*N*B*J + 8*M*M*F bytes).
 * Taps: L_n = floor(M/N) + (n < M mod N), each at most L, so that sum L_n = M
 * (the square model of Sec. II; M=4,6,8 with N=2 gives the paper's Table I).
 * EINVAL if a dimension is <= 0, N > M, M > CTFMNMF_MAX_M, B > CTFMNMF_MAX_B,
 * a derived L_n exceeds L, J <= max L_n, or out is NULL.
 * A bin's frames are processed by one thread block up to J = 4096 (M <= 4) or 1024
 * (M = 5..8); longer bins are split over a thread-block cluster of 2, 4 or 8 blocks that
 * combine their sums through distributed shared memory (two-kernel path, ISS update), up
 * to J = 32768 (M = 2) or 16384 (M = 3..8) and the device's shared memory.
 * EUNSUPPORTED if J exceeds those limits, or if the options ask for the persistent path
 * and the shape or the device does not allow it.
 * On success *out receives the handle; on failure *out is set to NULL.
 */
int ctfmnmf_create(int M, int N, int L, int B, int F, int J, ctfmnmf_t* out);

/* As ctfmnmf_create, with explicit taps Ln[N] (NULL: derived as above; sum must be M)
 * and options (NULL: defaults). dims->L only bounds the taps. */
int ctfmnmf_create_ex(const ctfmnmf_dims* dims, const int* Ln, const ctfmnmf_options* opt,
                      ctfmnmf_t* out);

/* Release every device buffer of h. h may be NULL. Synchronises h's stream first. */
int ctfmnmf_destroy(ctfmnmf_t h);

/* Short static description of the last failure on h (h NULL: last failed create on this
 * thread). Never NULL; "" if nothing failed. Valid until the next call on h. */
const char* ctfmnmf_last_error(ctfmnmf_t h);

/* Use stream (a cudaStream_t, NULL = legacy default stream) for all later work on h. */
int ctfmnmf_set_stream(ctfmnmf_t h, void* stream);

/* Write the taps L_n of h into Ln[N] (host). */
int ctfmnmf_get_taps(ctfmnmf_t h, int* Ln);

/*
 * Load the observed STFT X (device pointer, complex64 [M][F][J], read only during the
 * call's stream work) and reset the demixing state: W_i = I, y = x, log|det W_i| = 0
 * (initialisation of Sec. V-A). T and V are not changed: they keep the default init of
 * ctfmnmf_create, the values of ctfmnmf_set_init or the result of earlier iterations.
 * Synchronises the stream to check X:
 * ENONFINITE if X holds NaN or Inf (the state is then unusable until a good load).
 */
int ctfmnmf_load_stft(ctfmnmf_t h, const void* X);

/* As ctfmnmf_load_stft with X a host pointer (complex64 [M][F][J]); the copy to the
 * device is part of the call. Pinned memory gives the fastest copy. */
int ctfmnmf_load_stft_host(ctfmnmf_t h, const void* X);

/*
 * Set the NMF factors (device pointers, float32): T0 [N][F][B] (bases b_{n,i,k}) and
 * V0 [N][B][J] (activations v_{n,k,j}); values are floored at 1e-12. Either may be
 * NULL to keep the current value. Without this call, T and V start from the default
 * init: element e (flat C-order index) of T0 is 0.1 + 0.9*u(2e), of V0 0.1 + 0.9*u(2e+1),
 * u(c) = top 24 bits of splitmix64(seed * 2^32 + c) / 2^24, seed 0.
 * Synchronises the stream to check the values: ENONFINITE if any is NaN or Inf.
 */
int ctfmnmf_set_init(ctfmnmf_t h, const float* T0, const float* V0);

/*
 * Run n_iter >= 0 iterations (Sec. III): for each frequency bin the ISS sweep over the
 * M extended rows (Eqs. 11-16), the basis MU (Eq. 17), then the activation MU over all
 * bins (Eq. 18), then the scale normalisation (Eqs. 19-21). Asynchronous.
 * ESTATE if no STFT has been loaded.
 */
int ctfmnmf_iterate(ctfmnmf_t h, int n_iter);

/*
 * Wait for all work enqueued on the handle's stream and report device-side failures:
 * CTFMNMF_ETIMEOUT if a bounded device wait ran out since the last report (the solver
 * state is then undefined until the next ctfmnmf_load_stft), CTFMNMF_ECUDA on a CUDA error.
 */
int ctfmnmf_synchronize(ctfmnmf_t h);

/*
 * Negative log-likelihood of Eq. 5 without its constant, at the current state:
 * sum over bins, rows r=(n,l) and frames j >= l of log lambda_{n,i,j-l} +
 * |y_{r,i,j}|^2 / lambda_{n,i,j-l}, minus 2 J sum_i log|det W_i|.
 * Writes one double to *out (host). Synchronises the stream.
 */
int ctfmnmf_cost(ctfmnmf_t h, double* out);

/*
 * Source images by the multichannel Wiener filter of Eqs. 23-24; under the square model
 * it reduces to c_n = sum_l [W_i^{-1}]_{:,(n,l)} y_{(n,l),i,j}. Out: device pointer,
 * complex64 [N][M][F][J]. Asynchronous.
 */
int ctfmnmf_get_separated(ctfmnmf_t h, void* C);

/* As ctfmnmf_get_separated into a host buffer; synchronises the stream. */
int ctfmnmf_get_separated_host(ctfmnmf_t h, void* C);

/* Demixed extended rows y_{r,i,j} (Eq. 4): device pointer, complex64 [M][F][J]. */
int ctfmnmf_get_demixed(ctfmnmf_t h, void* Y);

/* Demixing matrices: device pointer, complex64 [F][M][M]; element [i][r][m] is the
 * coefficient of x_m in y_r, i.e. row r of W_i is w_r^H. */
int ctfmnmf_get_demix_matrix(ctfmnmf_t h, void* W);

/* log|det W_i| per bin, tracked through the determinant lemma: device pointer,
 * float64 [F]. */
int ctfmnmf_get_logdet(ctfmnmf_t h, double* logdet);

/* NMF factors: device pointers, float32 T [N][F][B] and V [N][B][J]; either may be NULL. */
int ctfmnmf_get_nmf(ctfmnmf_t h, float* T, float* V);

/*
 * Checkpoint/resume: restore a state exported with the getters above — Y [M][F][J]
 * complex64 (ctfmnmf_get_demixed), W [F][M][M] complex64 (ctfmnmf_get_demix_matrix),
 * T [N][F][B] and V [N][B][J] float32 (ctfmnmf_get_nmf), logdet [F] float64
 * (ctfmnmf_get_logdet); device pointers, read, none may be NULL. The handle then iterates
 * on from that state as the exporting handle would, to FP32 rounding (it forms 1/lambda
 * afresh from T and V). Synchronises the stream (the
 * rows are checked for NaN/Inf: ENONFINITE). The observation X is not part of the state:
 * a handle with the IP update keeps the X of its last ctfmnmf_load_stft and gives ESTATE
 * without one.
 */
int ctfmnmf_set_state(ctfmnmf_t h, const void* Y, const void* W, const float* T, const float* V,
                      const double* logdet);

/* ---- batched form: many mixtures advanced together ---- */

typedef struct ctfmnmf_batch* ctfmnmf_batch_t;

/*
 * Group `count` solver handles (all created on the current device, with equal v_update
 * and normalize options, each at most once) so that ctfmnmf_batch_iterate advances all of
 * them with shared launches: per iteration one bin-phase launch per class of mixtures with
 * equal template shape (M, frames per thread, block size), then one frame-phase launch per
 * class of base counts; the launches of n iterations are captured once into a CUDA graph
 * and replayed. The mixtures may differ in every dimension (ragged J, N, taps, B, F).
 * The handles keep owning their state: load_stft, set_init, cost and get_* stay per
 * handle; a handle must outlive the batch. The launch plan is chosen by an autotuner at
 * creation (it times two iterations of each candidate plan on the handles' buffers, saving
 * and restoring their state, so creating a batch changes no handle; it allocates and frees
 * temporary device memory of about the size of the mixtures' state). Work runs on the
 * stream of handles[0]. The candidate plans are numbered 2 * preference + merged (see
 * ctfmnmf_batch_info); as a diagnostic, the environment variable CTFMNMF_BATCH_PLAN=k (k in
 * 0..5) keeps only candidate k. Errors: EINVAL, ENOMEM, EUNSUPPORTED (no plan fits), ECUDA;
 * messages from ctfmnmf_last_error(NULL).
 */
int ctfmnmf_batch_create(int count, const ctfmnmf_t* handles, ctfmnmf_batch_t* out);

/* Run n_iter >= 0 iterations (as ctfmnmf_iterate) on every mixture of the batch;
 * asynchronous. ESTATE if a mixture has no STFT loaded. */
int ctfmnmf_batch_iterate(ctfmnmf_batch_t b, int n_iter);

/* Diagnostic: ctfmnmf_batch_iterate(b, n_iter) between two CUDA events on the batch's
 * stream; synchronises and writes the elapsed milliseconds to *ms (host). */
int ctfmnmf_batch_time(ctfmnmf_batch_t b, int n_iter, double* ms);

/* Diagnostic: info[5] (host) = {mixtures, bin classes, frame classes, chosen candidate
 * plan (2 * preference + merged-classes; preference 0: the single-mixture shape, 1: eight
 * strided frames per thread, 2: eight consecutive frames where the taps allow), kernels
 * launched so far}. */
int ctfmnmf_batch_info(ctfmnmf_batch_t b, int* info);

/*
 * Ragged buffers for the whole batch: one device buffer holding every mixture's block, and
 * offsets[k] (host array, in elements of the buffer's type) of mixture k's block.
 *   ctfmnmf_batch_load_stft:     X blocks [M][F][J] complex64 (as ctfmnmf_load_stft, each
 *                                checked for NaN/Inf; synchronises once).
 *   ctfmnmf_batch_set_init:      T0 blocks [N][F][B], V0 blocks [N][B][J] float32 (either
 *                                buffer may be NULL: that factor stays).
 *   ctfmnmf_batch_get_separated: images [N][M][F][J] complex64 (written, asynchronous).
 */
int ctfmnmf_batch_load_stft(ctfmnmf_batch_t b, const void* X, const long long* offsets);
int ctfmnmf_batch_set_init(ctfmnmf_batch_t b, const float* T0, const long long* t_offsets, const float* V0,
                           const long long* v_offsets);
int ctfmnmf_batch_get_separated(ctfmnmf_batch_t b, void* C, const long long* offsets);

/* Release the batch (not its handles). b may be NULL. */
int ctfmnmf_batch_destroy(ctfmnmf_batch_t b);

/* ---- differentiable form: gradients through the unrolled iterations ---- */

/*
 * A ctfmnmf_grad_t runs n_iter unrolled iterations (as ctfmnmf_iterate, default options:
 * all-taps activation update, normalisation) on a batch of S mixtures of one shape and
 * back-propagates a gradient given on the separated images (Eq. 24 in its projection-back
 * form, as ctfmnmf_get_separated) to the observations X and the initial factors T0, V0.
 * The paper differentiates nothing: the backward pass is the adjoint of every forward step
 * (ISS sweep Eqs. 11-16, basis MU Eq. 17, activation MU Eq. 18, normalisation Eqs. 19-21,
 * images Eq. 24) in reverse order, written by hand.
 * Gradient convention: for a real loss L and complex z = a + ib the gradient is
 * dL/da + i dL/db (PyTorch's). At a floor (T, V or lambda clamped) the gradient through
 * the clamped value is 0; a row with no energy (no normalisation) passes none through mu.
 * Memory: the state (Y, W, T, V) of every mixture is copied every ckpt_every iterations
 * during the forward pass (checkpoints), and the forward pass keeps the state before every
 * iteration of its last segment (ckpt_every slots, the tape). The backward pass reverses the
 * last segment from the tape and recomputes each earlier one from its checkpoint into the same
 * slots. ckpt_every >= n_iter: one segment, no recomputation, n_iter + 1 states in memory.
 * All device arguments are caller-owned; every call is asynchronous on the object's stream
 * unless stated. Error messages: ctfmnmf_last_error(NULL) on the calling thread.
 */
typedef struct ctfmnmf_grad* ctfmnmf_grad_t;

/* Create for `batch` >= 1 mixtures of shape dims with taps Ln[N] (NULL = derived from
 * dims->L as ctfmnmf_create), n_iter >= 1 iterations, a checkpoint every ckpt_every >= 1
 * iterations. EINVAL as ctfmnmf_create_ex; EUNSUPPORTED if M > 4, J > 2048 or B > 32;
 * ENOMEM. Allocates every buffer the forward and backward passes use. */
int ctfmnmf_grad_create(const ctfmnmf_dims* dims, const int* Ln, int batch, int n_iter, int ckpt_every,
                        ctfmnmf_grad_t* out);

/* All later work of g goes to this cudaStream_t (NULL = legacy default stream). */
int ctfmnmf_grad_set_stream(ctfmnmf_grad_t g, void* stream);

/* Forward pass: X [S][M][F][J] complex64, T0 [S][N][F][B], V0 [S][N][B][J] float32 (device,
 * read; floored at 1e-12 as ctfmnmf_set_init), C [S][N][M][F][J] complex64 (device, written):
 * the separated images after n_iter iterations from W = I. Inputs are not checked for NaN. */
int ctfmnmf_grad_forward(ctfmnmf_grad_t g, const void* X, const float* T0, const float* V0, void* C);

/* Backward pass of the last forward pass: gC [S][N][M][F][J] complex64 (device, read), the
 * gradient of the loss with respect to C. Writes gX [S][M][F][J] complex64, gT0 [S][N][F][B]
 * and gV0 [S][N][B][J] float32 (device). Each forward pass allows one backward pass (the
 * backward pass recomputes over the forward state); ESTATE otherwise. */
int ctfmnmf_grad_backward(ctfmnmf_grad_t g, const void* gC, void* gX, float* gT0, float* gV0);

/* Loss head: the mean over all S*N*M*F*J elements of |C - Cref|^2 (C, Cref [S][N][M][F][J]
 * complex64, device). If loss != NULL it is written to *loss (device double). If gC != NULL,
 * gC = scale * d(loss)/dC is written (device complex64), scale = *dloss (device double) or 1
 * when dloss is NULL. */
int ctfmnmf_grad_mse(ctfmnmf_grad_t g, const void* C, const void* Cref, double* loss, const double* dloss,
                     void* gC);

/* Diagnostic: kernels g has enqueued so far (forward and backward passes), to *count (host). */
int ctfmnmf_grad_launch_count(ctfmnmf_grad_t g, long long* count);

/* Release g and its buffers (synchronises its stream). g may be NULL. */
int ctfmnmf_grad_destroy(ctfmnmf_grad_t g);

/*
 * ctfmnmf_cost_noalloc -- the same negative log-likelihood as ctfmnmf_cost, computed from
 * caller-held buffers without allocating any device memory. The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc where they need the cost,
 * e.g. a real-time audio thread (an allocation may synchronise the device and has no
 * latency bound), code inside an allocator or memory-pool callback (it would re-enter the
 * allocator), or an application whose device memory is owned by another framework.
 *   Y [M][F][J] complex64, T [N][F][B] and V [N][B][J] float32, logdet [F] float64: device
 *   pointers in the layouts of ctfmnmf_get_demixed / _get_nmf / _get_logdet (read only);
 *   Ln[N]: host array of taps (sum M); out: device pointer to one double (written);
 *   stream: cudaStream_t (NULL = legacy default stream). Asynchronous.
 * Limit: F <= 16384 bins (EINVAL beyond, with a message from ctfmnmf_last_error(NULL)).
 * Scratch: the per-bin partial sums live in a 128 KiB static device array that every GPU
 * loading the library holds until exit. The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) and caches it; make that first call before any
 * stream capture. A device reset gives the device a new context, and the next call looks
 * the address up again. All calls share the array, and each call overwrites the slots it
 * uses: calls whose kernels overlap on the GPU (different streams or threads without
 * ordering) race and give wrong results.
 * Errors: EINVAL (dimensions, taps, null pointers, F too large), ECUDA (launch failed).
 */
int ctfmnmf_cost_noalloc(int M, int N, const int* Ln, int B, int F, int J, const void* Y,
                         const float* T, const float* V, const double* logdet, double* out,
                         void* stream);

/* ---- diagnostics (not part of the method) ---- */

/*
 * Run n_iter >= 1 iterations exactly like ctfmnmf_iterate but as plain stream launches
 * with a CUDA event pair around every launch, synchronise, and write to ms[2] (host) the
 * average device time in milliseconds of one launch of the bin-phase kernel (ISS sweep and
 * basis update, ms[0]) and of the frame-phase kernel (activation update and normalisation,
 * ms[1]). The state advances by n_iter iterations.
 */
int ctfmnmf_time_phases(ctfmnmf_t h, int n_iter, double* ms);

/* Number of kernels this handle has enqueued since it was created (host counter; a graph
 * replay counts every kernel node in it). Writes one int64 to *count (host). */
int ctfmnmf_get_launch_count(ctfmnmf_t h, long long* count);

/* Which path ctfmnmf_iterate takes for this handle: CTFMNMF_PATH_TWO_KERNEL or
 * CTFMNMF_PATH_PERSISTENT, written to *path (host). */
int ctfmnmf_get_path(ctfmnmf_t h, int* path);

/* The two-kernel bin phase's frames per thread and threads per block for this handle (both
 * 0 when its bins run over thread-block clusters), written to *fpt and *threads (host). */
int ctfmnmf_get_bin_shape(ctfmnmf_t h, int* fpt, int* threads);

/*
 * Persistent path only: run one launch of n_iter >= 1 iterations with a CUDA event pair
 * around the persistent kernel and another around the closing normalisation kernels;
 * synchronise; write the two durations in milliseconds to ms[2] (host). The state
 * advances by n_iter iterations. EUNSUPPORTED if the handle uses the two-kernel path.
 */
int ctfmnmf_time_persistent(ctfmnmf_t h, int n_iter, double* ms);

/*
 * Test hook for the bounded device waits: at the next persistent launch, thread block
 * `cta` does not arrive at the first grid barrier, so every other block's wait runs out
 * after wait_timeout_ms and the launch ends; ctfmnmf_synchronize then returns
 * CTFMNMF_ETIMEOUT and the state must be reloaded (ctfmnmf_load_stft). cta < 0 clears it.
 */
int ctfmnmf_debug_skip_arrival(ctfmnmf_t h, int cta);

/*
 * Debug builds (compiled with -DCTFMNMF_DEBUG): every kernel checks the indices it takes from
 * its launch (bin, frame tile, the batched form's work lists) against the shape before any
 * memory access; a failed check records itself in a device status word and the block returns,
 * and the next synchronising call on an affected handle returns CTFMNMF_EBOUNDS. This test hook
 * overwrites entry `entry` of bin class `cls`'s work list of batch b with (mixture, bin) so that
 * a test can watch such a check stop a block. Release builds return CTFMNMF_EUNSUPPORTED and
 * change nothing (their kernels do not check). *is_debug (host, may be NULL) receives 1 in a
 * debug build, else 0.
 */
int ctfmnmf_debug_set_work(ctfmnmf_batch_t b, int cls, int entry, int mixture, int bin, int* is_debug);

#ifdef __cplusplus
}
#endif
#endif /* CTFMNMF_H */
