/*
 * tucker_stream.h -- C ABI of the GB300 streaming ST-HOSVD library.
 *
 * Method: De, Li, Kolla, Phipps, "Efficient Computation of Tucker Decomposition for Streaming
 * Scientific Data Compression" (arXiv 2308.16395).
 *
 * Terms used below (paper notation):
 *   d        number of tensor modes, the streaming (time) mode last (Sec. 2.4); d-1 spatial modes.
 *   n_k      size of spatial mode k (fixed for the stream); a slice Y is n_1 x ... x n_{d-1}.
 *   r_k      Tucker rank of mode k; r_d is the streaming-mode rank.
 *   n_d      number of slices assimilated so far (rows of the streaming factor U_d).
 *   tau      relative error tolerance; every call keeps ||X - X^||_F <= tau ||X||_F (Alg. 5).
 *
 * Layouts: every tensor crossing this ABI is dense and column-major (mode 1 fastest), the
 * matricization convention of Sec. 2.1. A row-major array of shape (n_{d-1}, ..., n_1) has the
 * same bytes. Factor matrices are column-major n_k x r_k.
 *
 * Pointers named *_dev are CUDA device pointers on the current device; pointers named *_host are
 * host pointers. `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *
 * Ownership: the caller owns every buffer it passes and must keep input buffers unchanged until
 * the work enqueued on `stream` has completed; the library only reads inputs. The library owns
 * the tucker_state and all device memory behind it (released by tucker_destroy).
 *
 * Errors: argument errors (NULL pointers, d outside 2..8, sizes, tau <= 0, capacities) are
 * returned synchronously and leave the state unchanged. Conditions detected on the device
 * (a rank or size capacity exceeded, a non-finite slice norm, an eigensolver that did not
 * converge) are latched in the state and returned by the next call that synchronizes
 * (tucker_error_norm, tucker_get_ranks, tucker_get_step_info, tucker_copy_*); after that the
 * state accepts only tucker_destroy and the query calls. tucker_last_error gives a message.
 *
 * Threading: a state may be used from one host thread at a time. Calls on different states are
 * independent.
 */
#ifndef TUCKER_STREAM_H
#define TUCKER_STREAM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TUCKER_MAX_MODES 8

typedef struct tucker_state tucker_state; /* opaque, library-owned */

typedef enum {
  TUCKER_OK = 0,
  TUCKER_EINVAL = 1,     /* bad argument */
  TUCKER_ENOMEM = 2,     /* device allocation failed */
  TUCKER_ECAPACITY = 3,  /* a rank, the spatial core size or n_d outgrew its capacity */
  TUCKER_ENUMERIC = 4,   /* non-finite slice norm or eigensolver failure */
  TUCKER_ETIMEOUT = 5,   /* a bounded device wait gave up */
  TUCKER_ECUDA = 6,      /* a CUDA runtime call failed */
  TUCKER_ESTATE = 7      /* state unusable after an earlier latched error */
} tucker_status;

/* Slice element types. */
enum { TUCKER_F32 = 0, TUCKER_F64 = 1 };

/* Arithmetic forms.
 * TUCKER_PREC_FP64 : every step in FP64 (the plain method).
 * TUCKER_PREC_MIXED: slice-sized contractions (TTM chain, residual Grams, core and V updates) on
 *   FP32 data with FP32-accurate products; FP64 for norms and the error budget, eigen- and
 *   secular solves, rank truncation, the factors U_1..U_d, S, and the re-orthogonalisation of
 *   augmented factors. */
enum { TUCKER_PREC_FP64 = 0, TUCKER_PREC_MIXED = 1 };

typedef struct {
  int32_t ndim;                         /* d, 2..8 (spatial modes + the streaming mode) */
  int32_t dtype;                        /* TUCKER_F32 or TUCKER_F64: element type of slices */
  int32_t precision;                    /* TUCKER_PREC_FP64 or TUCKER_PREC_MIXED */
  int32_t block_cap;                    /* most slices one tucker_stream_update_block call takes,
                                           0..64 (0 = 1); the D* work buffers are allocated at
                                           creation for this many slices */
  int64_t n[TUCKER_MAX_MODES];          /* n_1..n_{d-1}; entries >= d-1 ignored */
  int64_t rank_cap[TUCKER_MAX_MODES];   /* capacity of r_1..r_d (0 = default: n_k for spatial
                                           modes, 256 for the streaming mode); r_d cap <= 512,
                                           spatial caps <= n_k, n_k <= 512 */
  int64_t steps_cap;                    /* capacity of n_d (rows of U_d) */
  int64_t core_cap;                     /* capacity of r_1*...*r_{d-1} (0 = product of caps) */
  double tau;                           /* relative tolerance tau > 0 (Sec. 2.3, Alg. 5) */
  double eps_m;                         /* orthogonality threshold of Alg. 3 (0 = 1e-10) */
} tucker_config;

/* Per-update decisions of the last tucker_stream_update (Alg. 4, Alg. 3). */
typedef struct {
  double eps;                           /* eps = tau ||Y|| / sqrt(d) (Alg. 5) */
  double y_norm2;                       /* ||Y||_F^2 */
  double e_norm2[TUCKER_MAX_MODES];     /* ||E_k||_F^2 of each spatial mode (Alg. 4) */
  int32_t grew[TUCKER_MAX_MODES];       /* 1 if ||E_k|| > eps (the factor was augmented) */
  int32_t r_add[TUCKER_MAX_MODES];      /* r'_k added to mode k */
  double q;                             /* ||e|| of the incremental SVD (Alg. 3) */
  int32_t augmented;                    /* 1 if q > eps (a new streaming basis vector) */
  int32_t r_stream;                     /* streaming rank after the update */
  double discarded;                     /* squared error added by this update (Prop. 1, 2) */
} tucker_step_info;

/* Batch ST-HOSVD (Alg. 2) of the first n_init slices X_dev (n_1 x ... x n_{d-1} x n_init,
 * column-major, element type cfg->dtype) with eps = tau ||X|| / sqrt(d), followed by the core
 * factorization C = V x_d S of Assumption 1(c). Creates *out. Synchronizes `stream`.
 * Errors: EINVAL (arguments, n_init < 1, X all zero), ENOMEM, ECAPACITY (a rank above its cap),
 * ENUMERIC, ECUDA. */
tucker_status tucker_init_sthosvd(const tucker_config* cfg, const void* X_dev, int64_t n_init,
                                  void* stream, tucker_state** out);

/* Streaming ST-HOSVD update (Alg. 5): assimilate one slice Y_dev (n_1 x ... x n_{d-1},
 * column-major, cfg->dtype). Spatial modes are updated by Alg. 4 (projection, residual,
 * residual Gram eigendecomposition, augmentation), the streaming mode by the incremental SVD
 * of Alg. 3, then the core is updated. Enqueued on `stream` without host synchronization; every
 * data-dependent branch is taken on the device. Errors: EINVAL, ESTATE (synchronous); device-side
 * conditions are latched (see above). */
tucker_status tucker_stream_update(tucker_state* s, const void* Y_dev, void* stream);

/* Host-input form of tucker_stream_update, for slices that arrive in host memory: copies Y_host
 * (same layout, preferably pinned) into one of two library-owned device staging buffers on an
 * internal copy stream, then enqueues the update of Y on `stream` after that copy. Returns
 * without waiting, so the next call's copy (into the other buffer) overlaps this update; a
 * buffer is reused only once the update that read it has completed. The caller keeps Y_host
 * unmodified until the copy has completed: at the latest when `stream` has reached this update.
 * From pageable memory the copy is synchronous for the caller. The staging buffers (2 slices)
 * are allocated on the first call. Errors: as tucker_stream_update; ENOMEM; ECUDA. */
tucker_status tucker_stream_update_host(tucker_state* s, const void* Y_host, void* stream);

/* Batched form: many independent streams, each updated by Alg. 5, advanced together by one
 * CUDA-graph launch per time step.
 *
 * tucker_batch_create captures one tucker_stream_update of every state into one CUDA graph, one
 * branch per state, so the updates of different streams run concurrently on the device. The
 * graph reads state i's next slice from the caller-owned device buffer Y_slots_dev[i] (layout and
 * type of that state's config), at every tucker_batch_update: the caller writes each time step's
 * slices into the slots (e.g. a simulation writes them there, or a host copy lands there), then
 * calls tucker_batch_update. Each update's device-side branches and ranks stay per state. The
 * states may differ in d, sizes, tau, dtype and precision; a state appears at most once.
 * Synchronizes each state's last stream once; enqueues no work.
 * Errors: EINVAL (NULL, count outside 1..4096, a repeated state), ESTATE (a state holds a latched
 * error), ECUDA (capture or instantiation failed). The states must outlive the batch; the slots
 * must stay allocated while it is used. tucker_stream_update may still be called on a state
 * between batch launches (on any stream; the caller orders the two). */
typedef struct tucker_batch tucker_batch;
tucker_status tucker_batch_create(tucker_state* const* states, const void* const* Y_slots_dev,
                                  int32_t count, tucker_batch** out);

/* One update of every state of the batch (one graph launch on `stream`, no host synchronization).
 * Device-side errors latch in the state that met them (the other states proceed) and are
 * reported by that state's next synchronizing call. Errors: EINVAL, ESTATE, ECUDA. */
tucker_status tucker_batch_update(tucker_batch* b, void* stream);

/* Kernel launches (graph kernel nodes) per tucker_batch_update; -1 for NULL. */
int64_t tucker_batch_kernels(const tucker_batch* b);

/* Release the graph (the states are not touched). */
void tucker_batch_destroy(tucker_batch* b);

/* One update (Alg. 5) of each of `count` independent states, state i from the slice Y_dev[i]
 * (device pointer; layout and type of that state's config), as one CUDA-graph launch on
 * `stream`. The first call for a given list of states captures the batch graph once (as
 * tucker_batch_create does; the call synchronizes the states' last streams then); later calls
 * with the same list, in the same order, write each state's slice address into its control
 * block (one small kernel per state on `stream`) and launch that graph. Slice pointers may
 * differ from call to call. A state appears at most once per list; destroying a state drops
 * the graphs that hold it. Calls with different lists keep separate graphs. The caller keeps
 * each slice unmodified until `stream` has passed this call. Device-side errors latch in the
 * state that met them. Errors: EINVAL (NULL, count outside 1..4096, a repeated state, a slice
 * unusable for TMA), ESTATE, ECUDA. */
tucker_status tucker_stream_update_batched(tucker_state* const* states, const void* const* Y_dev,
                                           int32_t count, void* stream);

/* Reconstruction X^(:, ..., t) = C x_1 U_1 ... x_{d-1} U_{d-1} x_d U_d(t, :) for slices
 * t in [t_begin, t_end) (0-based) into out_dev (n_1 x ... x n_{d-1} x (t_end - t_begin),
 * column-major, element type cfg->dtype). Enqueued on `stream`. Errors: EINVAL, ESTATE. */
tucker_status tucker_reconstruct(tucker_state* s, int64_t t_begin, int64_t t_end,
                                 void* out_dev, void* stream);

/* Allocation-free form of tucker_reconstruct. The paper has no counterpart: this entry point exists
 * for callers that cannot allocate device memory at the time they reconstruct. Examples are a
 * process whose device memory is already reserved in full by another allocator, code on a
 * device or under a virtualisation layer without stream-ordered memory pools (cudaMallocAsync,
 * which tucker_reconstruct uses, is unsupported there), and latency-critical loops that must not
 * pay for an allocation. Arguments, layout, output and errors are those of tucker_reconstruct.
 * The temporaries live in one fixed device array of TUCKER_NOALLOC_SCRATCH_BYTES, which every GPU
 * that loads this library holds until the process exits; each of the two temporaries may use
 * half of it. A call whose largest temporary, C x_d U_d(t_begin:t_end, :) or a partial expansion
 * C x_d U_d x_1 U_1 ... x_k U_k (k < d-1), needs more than half returns TUCKER_EINVAL before
 * any device work. Reconstruct fewer slices per call in that case. The call allocates nothing:
 * no cudaMalloc, no cudaFree, no pool or library allocation. Every call looks up the array's
 * device address in the current device's context (cudaGetSymbolAddress, which allocates
 * nothing); the first lookup in a context also loads the library's device symbols, so make the
 * first call on each device outside any stream capture. Every call, on every state, shares the one array and
 * keeps its last contents. Nothing in it needs to start at zero, because each call writes every
 * element it reads. Calls whose device work overlaps (on different streams or host threads)
 * race on the array and must be serialised by the caller. Synchronizes `stream` once before
 * its launches, to read the ranks. */
#define TUCKER_NOALLOC_SCRATCH_BYTES (16 * 1024 * 1024)
tucker_status tucker_reconstruct_noalloc(tucker_state* s, int64_t t_begin, int64_t t_end,
                                         void* out_dev, void* stream);

/* Running error bound and data norm (Prop. 1, Prop. 2, App. D): *err_bound_host is the square
 * root of the accumulated squared truncation error (initial ST-HOSVD + every update), an upper
 * bound of ||X - X^||_F; *data_norm_host = ||X||_F over every slice seen. Synchronizes. */
tucker_status tucker_error_norm(tucker_state* s, double* err_bound_host, double* data_norm_host);

/* Asynchronous form of tucker_error_norm for pipelined callers: enqueues on `stream` a copy of
 * the squared running error bound and the squared data norm, as they stand after the work
 * enqueued so far, into out2_host[0] and out2_host[1] (host memory, preferably pinned). With
 * pinned (mapped) or managed memory a one-thread kernel stores the values, so the read does not
 * wait in a copy-engine queue behind host-to-device copies of other streams; other memory is
 * copied by cudaMemcpyAsync. No synchronization: the values are valid once `stream` has reached
 * this point. A latched device error is not reported here (the next synchronizing call reports
 * it). Errors: EINVAL, ESTATE, ECUDA. */
tucker_status tucker_error_norm_async(tucker_state* s, double* out2_host, void* stream);

/* Current ranks r_1..r_d (d entries) and n_d. Synchronizes. */
tucker_status tucker_get_ranks(tucker_state* s, int64_t* ranks_host, int64_t* n_d_host);

/* Decisions of the most recent update. Synchronizes. */
tucker_status tucker_get_step_info(tucker_state* s, tucker_step_info* info_host);

/* Per-update log (Alg. 5 decisions). Every update since the initial ST-HOSVD leaves one record
 * in a device array of steps_cap records (written by the update's last kernel, so recording
 * costs no synchronization); tucker_get_step_log copies records [first, first + count) (0 = the
 * first update after tucker_init_sthosvd) into out_host. The tails are Alg. 1's sums of the
 * discarded eigenvalues of a grown mode's residual Gram at the chosen cut r'_k (tail_cut, the
 * squared error that mode's truncation adds) and at r'_k - 1 (tail_prev, above eps^2 by the cut
 * rule unless the cut was forced). Synchronizes. Errors: EINVAL (range beyond the updates
 * recorded), latched device errors. */
typedef struct {
  int64_t n_d;                              /* n_d after the update */
  int32_t ranks[TUCKER_MAX_MODES];          /* r_1..r_d after the update */
  int32_t grew[TUCKER_MAX_MODES];           /* spatial mode k grew: ||E_k|| > eps (Alg. 4) */
  int32_t r_add[TUCKER_MAX_MODES];          /* r'_k */
  int32_t eig_path[TUCKER_MAX_MODES];       /* grown mode: 1 = subspace iteration + FP64
                                               Rayleigh-Ritz cut, 2 = full tridiagonal solver */
  int32_t eig_iters[TUCKER_MAX_MODES];      /* grown mode, path 1: subspace iterations */
  int32_t augmented;                        /* q > eps (Alg. 3) */
  int32_t replayed;                         /* 1 if tucker_replay_next forced this update */
  double eps;                               /* tau ||Y|| / sqrt(d) */
  double y_norm2;                           /* ||Y||^2 */
  double e_norm2[TUCKER_MAX_MODES];         /* ||E_k||^2 */
  double tail_cut[TUCKER_MAX_MODES];        /* grown mode: tail of the eigenvalues at r'_k */
  double tail_prev[TUCKER_MAX_MODES];       /* grown mode: tail at r'_k - 1 */
  double q;                                 /* ||e|| (Alg. 3) */
  double discarded;                         /* squared error added by this update */
} tucker_step_record;
tucker_status tucker_get_step_log(tucker_state* s, int64_t first, int64_t count,
                                  tucker_step_record* out_host);

/* Decision replay: a TEST HOOK, not part of the method. Under mixed precision a decision whose
 * statistic lies within a small relative distance of eps^2 (||E_k||^2 in Alg. 4, an eigenvalue
 * tail at the cut of Alg. 1, q^2 in Alg. 3) can come out differently from an FP64 computation
 * of the same step; once it has, the two states follow different paths and can no longer be
 * compared. This call forces the decisions of the NEXT update (tucker_stream_update,
 * tucker_stream_update_host or tucker_batch_update) of state s, so that a test can make the
 * library take a reference's decision at such a step and keep comparing afterwards.
 * grow[k] (k < d-1): -1 keeps the update's own decision for spatial mode k, 0 forces
 * ||E_k|| <= eps (no growth), r > 0 forces growth with r'_k = r (clamped to n_k - r_k);
 * augment: -1 keeps Alg. 3's own branch, 0 forces q <= eps, 1 forces q > eps (ignored when
 * e = 0). The forced values reach the device with the next update, on its stream; the update
 * that used them is marked in its log record. Synchronizes the state's last stream.
 * Errors: EINVAL (NULL, values out of range), ESTATE, ECUDA. */
typedef struct {
  int32_t grow[TUCKER_MAX_MODES];
  int32_t augment;
} tucker_replay;
tucker_status tucker_replay_next(tucker_state* s, const tucker_replay* r);

/* Orthogonality of the factors: out_host[k] = ||U_k^T U_k - I||_F for k = 0..d-1 (U_d the
 * streaming factor, n_d x r_d), computed in FP64 on the device. Sec. 3.1 remarks that forming the
 * new left singular vectors of the incremental SVD (Alg. 3) as a product U' U'' may lose
 * orthogonality over many updates; this measures it. Synchronizes.
 * Errors: EINVAL (NULL), ENOMEM, ESTATE, ECUDA. */
tucker_status tucker_orthogonality_error(tucker_state* s, double* out_host);

/* Restores the orthonormality of the streaming factor: U_d is replaced by its polar factor (the
 * nearest matrix with orthonormal columns), computed by two Newton-Schulz steps
 * U <- U (3 I - U^T U) / 2 in FP64 on the device. C, S and V are kept (Assumption 1 is
 * untouched); the reconstruction moves by (U_d' - U_d) C_(d), whose norm ||(U_d' - U_d) S||_F
 * is added to the running error bound (triangle inequality) and returned in *change_host (may be
 * NULL). Meant for long streams, every few thousand updates or when tucker_orthogonality_error
 * reports a deviation well above rounding. Allocates and frees temporary device memory.
 * Synchronizes. Errors: EINVAL (NULL), ENOMEM, ESTATE, ECUDA. */
tucker_status tucker_restore_orthogonality(tucker_state* s, void* stream, double* change_host);

/* Block update: assimilate nslices slices at once (Y_dev: nslices slices, each n_1 x ... x n_{d-1}
 * column-major, stored one after the other; device memory, caller-owned, read during the call's
 * kernels). The paper names processing several slices at once as future work (Conclusions).
 * The spatial modes take the block as one tensor with a trailing mode of size nslices: Alg. 4
 * for each mode with eps = tau ||Y_block|| / sqrt(d), so one residual pass, one Gram and one
 * rank cut per mode cover the whole block. The streaming mode then takes the nslices projected
 * slices as new rows, one incremental-SVD step (Alg. 3) each in slice order, with the tolerance
 * eps / sqrt(nslices) per row: the block adds at most (d - 1) eps^2 + nslices eps^2 / nslices =
 * tau^2 ||Y_block||^2 to the squared error, Alg. 5's guarantee for the block. nslices = 1 is
 * tucker_stream_update. n_d grows by nslices; the step log gets one record per slice (the
 * block's spatial decisions and norm in the first). nslices must not exceed the configuration's
 * block_cap. Without phase profiling the first block of each size is captured as a CUDA graph
 * (the form of tucker_stream_update, with the block's rows unrolled) and later blocks of that
 * size launch it; with profiling on, blocks run launch by launch. The slices' address must be
 * 16-byte aligned for the tensor-core pass (EINVAL otherwise).
 * Errors: EINVAL (NULL, nslices < 1 or above block_cap), ESTATE, ECUDA; device errors
 * (ECAPACITY, ENUMERIC, ETIMEOUT) latch and surface at the next synchronizing call. */
tucker_status tucker_stream_update_block(tucker_state* s, const void* Y_dev, int32_t nslices,
                                         void* stream);

/* Test hook of the bounded waits: the next update's mode-1 tensor-core pass (mixed form, FP32
 * slices, n_1 <= 384) withholds its loads, so every wait of the kernel's consumers gives up after
 * its time limit (1 s of wall time). The kernel then latches TUCKER_ETIMEOUT and ends normally:
 * the update's later kernels return at once, the next synchronizing call returns ETIMEOUT, the
 * state is unusable afterwards (ESTATE) and the CUDA context stays usable. No fault, trap or
 * unbounded wait is involved. Synchronizes the state's last stream.
 * Errors: EINVAL (NULL), ESTATE, ECUDA. */
tucker_status tucker_test_stall_next(tucker_state* s);

/* Re-compression of the streamed decomposition: the batch ST-HOSVD (Alg. 2) run again on the
 * current Tucker representation X^ = C x_1 U_1 ... x_d U_d, so that ranks the per-slice updates
 * over-estimated come down. Since the factors are orthonormal, Alg. 2 on X^ equals Alg. 2 on the
 * core C (r_1 x ... x r_d, the streaming mode's r_d entries taken as its slices) followed by
 * U_k <- U_k Q_k, with Q_k the factors of the core's decomposition; the new core, S and V come
 * from that decomposition's last mode (C' = V' x_d S', Assumption 1(c)).
 * Budget: with b the running bound (sqrt of the accumulated discarded energy) and ||X|| the
 * norm of the data seen so far, the core's decomposition takes the per-mode tolerance
 * eps' = (tau_total ||X|| - b) / sqrt(d), so that its discarded energy e' <= (tau_total ||X|| -
 * b)^2; the new bound is (b + sqrt(e'))^2 (triangle inequality), hence ||X - X^'|| <=
 * tau_total ||X||. Streaming continues from the new state with the configured tau.
 * tau_total must exceed b / ||X||. The core's decomposition runs in FP64 on the device
 * (spatial ranks <= 256); temporary device memory is allocated and freed. Synchronizes.
 * info (host, may be NULL) receives the new ranks, the core decomposition's discarded energy e'
 * and the new bound.
 * Errors: EINVAL (NULL, tau_total <= b / ||X||, a spatial rank above 256), ENOMEM, ESTATE,
 * ECUDA, and the errors of tucker_init_sthosvd. */
typedef struct {
  int64_t ranks[TUCKER_MAX_MODES];  /* r'_1..r'_d; entries >= d are 0 */
  double discarded;                 /* e' (energy the core's truncation dropped) */
  double err_bound;                 /* b + sqrt(e'), the new running bound */
} tucker_recompress_info;
tucker_status tucker_recompress(tucker_state* s, double tau_total, void* stream,
                                tucker_recompress_info* info);

/* Copy U_k (mode = 0..d-1, 0-based) as FP64 column-major (rows x r_k) into dst_dev, where rows
 * is n_k for spatial modes and n_d for the streaming mode. Synchronizes. */
tucker_status tucker_copy_factor(tucker_state* s, int32_t mode, double* dst_dev);

/* Copy the core C (r_1 x ... x r_d, FP64, column-major) into dst_dev. Synchronizes. */
tucker_status tucker_copy_core(tucker_state* s, double* dst_dev);

/* Copy S (r_d values, FP64) and V (r_1 x ... x r_d, FP64, column-major; V_(d) row-orthonormal,
 * C = V x_d S when the last residual was kept, Assumption 1(c)) into device buffers. Either
 * pointer may be NULL. Synchronizes. */
tucker_status tucker_copy_sv(tucker_state* s, double* S_dev, double* V_dev);

/* Profiling (tracing) of the update phases. Phase indices: 0 mode-1 projection + residual norm
 * (the pass over the slice), 1 projections of modes 2..d-1, 2 growth work (residual Gram, eigen-
 * solve, augmentation, re-projection), 3 incremental-SVD passes and the secular SVD, 4 streaming
 * factor update and M, 5 core and V updates. */
#define TUCKER_NPHASES 6
typedef struct {
  double ms[TUCKER_NPHASES];     /* CUDA-event time per phase, summed over profiled updates */
  double bytes[TUCKER_NPHASES];  /* algorithmic bytes per phase (operands read/written once per
                                    pass, from the ranks in effect), summed */
  int64_t launches;              /* kernels launched by profiled updates */
  int64_t updates;               /* profiled updates */
  double ms_slice_pass;          /* CUDA-event time of the launch that streams the slice (the
                                    mode-1 projection + residual kernel alone), summed */
} tucker_profile;

/* on = 1: the following updates record CUDA events around each phase on their stream (adds
 * event records, no synchronization); on = 0: stop. Resets the accumulated profile. */
tucker_status tucker_profile_enable(tucker_state* s, int32_t on);

/* Accumulated profile since tucker_profile_enable. Synchronizes. */
tucker_status tucker_profile_read(tucker_state* s, tucker_profile* out_host);

/* Execution form of tucker_stream_update. Without phase profiling, the first update of a state
 * captures the update as a CUDA graph: every data-dependent branch stays on the device, each
 * spatial mode's growth chain (residual Gram, eigensolve, augmentation, re-projection) becomes a
 * conditional IF node whose condition the device sets from ||E_k|| > eps, and each later call
 * writes the slice address (and its TMA descriptor) into the state with one small host-to-device
 * copy and launches the graph. With profiling on, updates are issued as individual launches.
 * Returns the kernel nodes of the captured update graph (conditional bodies included: an upper
 * bound of the kernels one update runs), 0 before the first capture, -1 for NULL. */
int64_t tucker_graph_kernels(const tucker_state* s);

/* Kernel nodes of the captured graph of a block update of nslices slices (conditional bodies
 * included), 0 before that size's first block, -1 for NULL or nslices outside 2..64. */
int64_t tucker_block_graph_kernels(const tucker_state* s, int32_t nslices);

/* Launch shape of the update's kernels: CTA counts of its grid-stride passes. The defaults fill
 * the whole GPU (two CTAs per SM for the projection and ISVD passes, one per SM for the
 * tensor-core passes, four per SM for the core/V update); states updated concurrently (the batched
 * form) run faster with smaller shares, which bench.py's batched workload chooses with the
 * autotuner in paper_2308_16395_gb300/autotune.py. A plan changes no result, only how the work
 * is split. Zero fields keep the default. */
typedef struct {
  int32_t grid_proj;   /* SIMT projection / residual passes and norm partial sums, 1..4096 */
  int32_t grid_tc;     /* tensor-core passes (projection, E^T, Gram, core/V), 1..SM count */
  int32_t grid_isvd;   /* ISVD row passes, 1..304 */
  int32_t grid_cv;     /* core / V update, 1..65535 */
} tucker_launch_plan;

/* Set the plan. Takes effect at the next update (a captured update graph is discarded and
 * captured again); a batch must be created after its states' plans are set. Synchronizes the
 * state's last stream. Errors: EINVAL (field out of range), ESTATE. */
tucker_status tucker_set_launch_plan(tucker_state* s, const tucker_launch_plan* plan);

/* The plan in effect (defaults resolved). */
tucker_status tucker_get_launch_plan(const tucker_state* s, tucker_launch_plan* plan_host);

/* Message for the last error on this state (static storage owned by the state; never NULL). */
const char* tucker_last_error(const tucker_state* s);

/* Release the state and its device memory. Synchronizes the device work of the state. */
void tucker_destroy(tucker_state* s);

/* Library version string. */
const char* tucker_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TUCKER_STREAM_H */
