/*
 * cumwin — sliding-window cumulant tensors of orders 1..d on one GPU.
 *
 * C ABI of the library.  It follows the problem statement of Domino & Gawron,
 * "Algorithm for an arbitrary-order cumulant tensor calculation in a sliding
 * window of data streams":
 *   - a window X^(w) holds the last T samples of an n-variate stream, one
 *     sample per row (Section 2.1, Eqs. 1-4);
 *   - each shift drops the oldest p rows X_(-) and appends p new rows X_(+)
 *     (Algorithm 1), and the moment tensors of orders 1..d are updated by
 *     M(X^(w+1)) = M(X^(w)) + (p/T)(M(X_(+)) - M(X_(-))) (Eqs. 6-7, Algorithm 2);
 *   - the cumulant tensors C_1..C_d are recovered from the moments by the
 *     moment-to-cumulant relation (Algorithms 3-4);
 *   - their Frobenius norms and the non-Gaussianity estimator
 *     nu_s = ||C_s||_2 / ||C_2||_2^{s/2} are reduced (Eqs. me, mef, Algorithm 5).
 *
 * Storage: super-symmetric tensors of order s are kept in the block
 * ("hyper-pyramid") structure of Section 2.3: with nbar = ceil(n/b) blocks per
 * mode, only blocks j1 <= j2 <= ... <= js are stored, in lexicographic order of
 * (j1..js); each block is a dense b^s array, row-major over the in-block
 * indices (a1..as) with a1 slowest, and diagonal blocks are stored whole.
 * Element (block rank r, in-block offset o) lives at r * b^s + o and holds the
 * tensor entry at variables (j1*b+a1, ..., js*b+as).  When b does not divide n,
 * variables n..nbar*b-1 are zero padding and every entry that involves one of
 * them is exactly 0.
 *
 * Conventions for every call:
 *   - pointers named *_dev are CUDA device pointers owned by the caller; they
 *     must stay valid until the handle's stream has executed the call;
 *   - pointers named *_host are host pointers;
 *   - samples are FP32, row-major, row stride `ld` (>= n) in elements;
 *   - calls are asynchronous on the handle's stream unless stated otherwise;
 *   - argument errors are returned synchronously and leave the state
 *     unchanged; device-side conditions (a non-finite input sample) set a
 *     sticky status word that the next synchronising call reports;
 *   - a handle is not thread-safe: one host thread at a time.
 */
#ifndef CUMWIN_H
#define CUMWIN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cumwin_s* cumwin_t;

/* Return codes. */
enum {
    CUMWIN_OK = 0,
    CUMWIN_EINVAL = -1,     /* bad argument (sizes, order, null pointer)          */
    CUMWIN_ENOMEM = -2,     /* device allocation failed                           */
    CUMWIN_ECUDA = -3,      /* a CUDA runtime call failed (see cumwin_last_error) */
    CUMWIN_ESTATE = -4,     /* call out of sequence (e.g. push before fill)       */
    CUMWIN_ENONFINITE = -5, /* a non-finite sample entered the window             */
    CUMWIN_ETIMEOUT = -6,   /* a bounded device wait gave up                      */
    CUMWIN_ENOTSUP = -7     /* combination not supported on this device/build     */
};

/* Arithmetic of the moment-sum update (the cumulant recovery and all running
 * sums are FP64 in every form). */
enum {
    CUMWIN_FP64 = 0,        /* FP64 products and FP64 accumulation                 */
    CUMWIN_MIXED_BF16 = 1,  /* tensor cores: BF16 hi+lo split products (3 MMAs),
                               FP32 accumulation per batch, FP64 running sums     */
    CUMWIN_MIXED_FP16 = 2   /* as above with FP16 hi+lo splits                     */
};

/*
 * Device memory.  Every byte of device state a handle or a batch holds (ring
 * buffer, sums, cumulants, tables, workspaces, the scratch of every call) is
 * taken from an allocator when the handle is created (the adjoint's
 * workspace: at the first cumwin_grad) and given back when it is destroyed;
 * no other call allocates.  The paper has no counterpart (it states the
 * method on a window held in memory); the allocator only decides where that
 * memory comes from:
 *   alloc(ctx, bytes, stream, &ptr) returns 0 and a device pointer (aligned
 *     to at least 256 bytes) usable on every stream once it returns, or a
 *     nonzero value when it cannot (the library then reports ENOMEM);
 *   free(ctx, ptr, bytes, stream) gives it back; the library has synchronised
 *     its streams before it frees.
 * `stream` is the handle's stream at the time of the call.
 */
typedef int (*cumwin_alloc_fn)(void* ctx, size_t bytes, void* cuda_stream, void** out_dev);
typedef void (*cumwin_free_fn)(void* ctx, void* dev_ptr, size_t bytes, void* cuda_stream);

/* Process-wide allocator for handles and batches created from now on (each
 * keeps the allocator it was created with until it is destroyed).  Both NULL
 * restores the default: cudaMallocAsync on the handle's stream, synchronised,
 * and cudaFree.  Thread-safe.  Errors: EINVAL when only one is NULL. */
int cumwin_set_allocator(cumwin_alloc_fn alloc, cumwin_free_fn free_fn, void* ctx);

/* Bytes of device memory the handle holds (all taken from its allocator). */
int64_t cumwin_device_bytes(cumwin_t h);

/* Largest supported order d and variable count n. */
#define CUMWIN_MAX_ORDER 8
#define CUMWIN_MAX_N 256

/*
 * Create a handle for n variables, orders 1..d, block size b (1 <= b), window
 * length T samples, nominal shift size p (the paper's t_up, 1 <= p <= T),
 * arithmetic `precision`, issuing work on `cuda_stream` (a cudaStream_t;
 * NULL = legacy default stream).  Allocates all device state (ring buffer of
 * T samples, FP64 moment sums and cumulants of every order, tables, and the
 * batch-sum FIFO of cumwin_push when T is a multiple of p and it takes at most
 * a quarter of the free memory: T/p x sum_s E_s floats in the mixed forms,
 * doubles in the FP64 form) on the current device from the allocator of
 * cumwin_set_allocator.  Synchronous.
 * In the mixed forms the FP32 tile sums are formed per batch of p samples and
 * the first window is summed in batches of p aligned with the later shifts,
 * so when every push has p rows and p divides T a batch's FP32 sum leaving
 * the window is bitwise the one that entered it and the running FP64 sums do
 * not drift.  Pushes of another size are accepted.
 * Errors: EINVAL (n < 1, n > CUMWIN_MAX_N, d < 1, d > CUMWIN_MAX_ORDER, b < 1,
 * T < 1, p outside [1, T], unknown precision), ENOTSUP (mixed precision on a
 * device other than sm_103), ENOMEM, ECUDA.
 */
int cumwin_create(int n, int d, int b, int64_t T, int p, int precision, void* cuda_stream,
                  cumwin_t* out);

/*
 * Block shards of one stream over several GPUs (one handle per GPU, all fed the
 * same samples).  The stored blocks of the top order d, in lexicographic order
 * (Section 2.3), are split into nshards contiguous ranges of nearly equal block
 * count (cumwin_shard_blocks); shard `shard` updates (Eqs. 6-7) and recovers
 * (Algorithms 3-4) only the blocks of its range, and its squared norm of order
 * d is the sum over its blocks, so the norm of the whole tensor is the sum of
 * the shards' values (an all-reduce).  Orders below d are small and are kept
 * whole on every shard.  C_d and M_d read from a shard are valid inside its
 * block range only.  Not in the paper (it parallelises over sub-series of the
 * samples instead).  Needs a mixed form and d = 5 or 6 with b^d >= 256 for
 * nshards > 1 (ENOTSUP otherwise); cumwin_grad is not available on a shard.
 * cumwin_create is cumwin_create_shard with shard 0 of 1.
 */
int cumwin_create_shard(int n, int d, int b, int64_t T, int p, int precision, void* cuda_stream, int shard,
                        int nshards, cumwin_t* out);
/* Host only: the block range [*begin, *end) of order d owned by shard `shard` of `nshards`. */
int cumwin_shard_blocks(int n, int b, int d, int shard, int nshards, int64_t* begin, int64_t* end);
/* Host only: ||C_s|| = sqrt(fro2[s-1]) and nu_s (Eq. mef, NaN for s < 3) from the squared
 * norms of orders 1..d, e.g. after summing the shards' values; either output may be NULL. */
int cumwin_estimators_from_fro2(int d, const double* fro2_host, double* fro_host, double* nu_host);

/* Free all device state.  Synchronises the handle's stream first.  NULL is a no-op. */
int cumwin_destroy(cumwin_t h);

/* Change the stream later calls are issued on.  The new stream first waits
 * (on the device) for the work issued so far on the old stream and for any
 * pending pipelined recovery, so the handle's calls stay in order.  When either
 * stream is being captured, ordering the two streams is left to the capturer. */
int cumwin_set_stream(cumwin_t h, void* cuda_stream);

/*
 * Load the first window X^(1) (T rows, row stride ldx >= n, device) and compute
 * its moments, cumulants and norms in full (Algorithm 1, "calculate moments
 * M_1(X^(1))..M_d(X^(1))").  In the mixed forms this also fixes the shift
 * vector (the FP32-rounded column means of X^(1)) about which all moments are
 * accumulated; cumulants of order >= 2 do not depend on it.
 */
int cumwin_fill(cumwin_t h, const float* X_dev, int64_t ldx);

/*
 * One window shift (one pass of the loop of Algorithm 1): append the p rows of
 * x_in_dev (X_(+)), drop the p oldest rows (X_(-)), update the moment sums of
 * every order by sum_{in} x^{(x)s} - sum_{out} x^{(x)s} (Eqs. 6-7), recover
 * C_1..C_d (Algorithms 3-4) and reduce their norms on the device.
 * x_out_dev == NULL: X_(-) is taken from the ring buffer (Algorithm 1, "first
 * t_up rows of X^(w)").  Non-NULL: the caller supplies X_(-) (the inputs of
 * momentsupdate in Algorithm 2); the ring buffer is still advanced with x_in.
 * Requires 1 <= p <= T and a prior cumulant fill.  Errors: EINVAL, ESTATE.
 * Allocates nothing and does not synchronise (capturable into a CUDA graph).
 *
 * T a multiple of the nominal p: the handle keeps a FIFO of the T/p batch
 * sums (sum_s E_s each; FP32 in the mixed forms, FP64 in the FP64 form), the
 * alternative scheme of Section 2.4, filled by cumwin_fill / cumwin_recompute,
 * when it takes at most a quarter of the free device memory.  A shift of
 * exactly p rows with x_out_dev == NULL then subtracts the leaving batch's
 * stored sum instead of recomputing it (half the update's multiply-adds).  In
 * the mixed forms the result is bitwise the one of the recomputing form; in
 * the FP64 form it differs from it by the rounding of the FP64 additions (the
 * FIFO form subtracts the leaving batch's sum as a whole, the recomputing form
 * accumulates the leaving products into the entering batch's sum).  Any other
 * shift (x_out_dev != NULL or another number of rows) recomputes X_(-) and
 * retires the FIFO until the next fill or recompute.  A push captured into a
 * CUDA graph keeps the choice made at capture (cumwin_fifo tells which): after
 * an irregular shift outside the graph, call cumwin_recompute before replaying
 * a graph whose pushes use the FIFO.
 *
 * Pipelined shifts (mixed forms): the recovery of C_1..C_d and of the norms
 * runs on a stream owned by the handle, ordered after the shift's moment
 * update by an event, so that the next push's staging and tensor-core update
 * overlap it (the two alternate between two update workspaces).  Every other
 * entry point of the handle first makes the handle's stream wait for it, so
 * results read through the API are always those of the last push; work the
 * caller queues on the stream itself (e.g. a timing event after the push)
 * needs cumwin_join first.  A push issued under stream capture, or with
 * phase timing on, runs the recovery on the handle's stream.
 */
int cumwin_push(cumwin_t h, const float* x_in_dev, const float* x_out_dev, int p, int64_t ld);

/* Make the handle's stream wait (on the device; the host does not block) for
 * the recovery of the last pipelined push.  Always succeeds on a valid handle. */
int cumwin_join(cumwin_t h);

/*
 * Enqueue copies of the squared norms ||C_s||_F^2, s = 1..d (d doubles, into
 * fro2_out) and of the sticky device status (one int, into status_out) of the
 * window as it stands after the calls issued so far.  Either pointer may be
 * NULL, not both; each may be device memory or host memory (pinned for an
 * asynchronous copy).  After a pipelined push the copies run on the recovery
 * stream behind that push's recovery, so they do not hold back the next
 * push; otherwise on the handle's stream.  The values are in place once the
 * handle's stream has been synchronised after cumwin_join (or the device has
 * been synchronised).  Nothing is allocated; the host does not block.
 */
int cumwin_norms_enqueue(cumwin_t h, double* fro2_out, int* status_out);

/*
 * As cumwin_norms_enqueue, with the estimators formed on the device: the
 * Frobenius norms ||C_s||_F, s = 1..d (Eq. me, d doubles, into fro_out), the
 * non-Gaussianity estimators nu_s = ||C_s|| / ||C_2||^{s/2} (Eq. mef, d
 * doubles into nu_out, NaN for s < 3 and when ||C_2|| = 0) and the sticky
 * status (into status_out).  Any of the three may be NULL, not all; each may
 * be device or host memory.  Ordering and validity as cumwin_norms_enqueue;
 * nothing is allocated and the host does not block.
 */
int cumwin_estimators_enqueue(cumwin_t h, double* fro_out, double* nu_out, int* status_out);

/*
 * L = sum_{s=1..d} w[s] ||C_s||_F^2 of the current window (w_host: d+1
 * doubles, w[0] ignored; full-tensor norms, Eq. me) into L_dev[0] (device,
 * FP64).  Not in the paper: it is the scalar whose gradient cumwin_grad
 * evaluates.  Asynchronous on the handle's stream; w_host is read before the
 * call returns.  Errors: EINVAL, ESTATE.
 */
int cumwin_loss(cumwin_t h, const double* w_host, double* L_dev);

/* Turn pipelined shifts (cumwin_push) on (enable != 0, the default) or off.
 * Results are bitwise the same either way. */
int cumwin_set_pipeline(cumwin_t h, int enable);

/* 1 when the next shift of the nominal p rows (x_out_dev == NULL) will use
 * the batch-sum FIFO of cumwin_push, 0 when it recomputes X_(-) (T not a
 * multiple of p, no room for the FIFO, or it was retired), EINVAL. */
int cumwin_fifo(cumwin_t h);

/*
 * As cumwin_push with X_(+) in HOST memory (pinned memory gives an
 * asynchronous copy; pageable memory makes the copy synchronous).  The copy
 * goes to one of two device staging buffers owned by the handle, on a copy
 * stream of the handle, so that it overlaps the kernels of the previous
 * pushes; the push waits for its copy, and a buffer is reused only after the
 * push that read it.  Under stream capture the copy runs on the handle's stream.
 */
int cumwin_push_host(cumwin_t h, const float* x_in_host, int p, int64_t ld);

/* Copy C_s (1 <= order <= d) of the current window, block layout, FP64,
 * cumwin_layout_size(n, b, order) elements, into out_dev. */
int cumwin_cumulants(cumwin_t h, int order, double* out_dev);

/* Expand C_s (1 <= order <= d) of the current window into the full
 * n^order tensor, row-major over (i_1, ..., i_order) with every permutation of
 * a sorted index tuple holding the same value (the super-symmetric tensor the
 * block layout of Section 2.3 stores once), FP64, n^order doubles into
 * out_dev.  Order 1 includes the shift (it is the window mean).  Errors:
 * EINVAL (also when n^order exceeds 2^36), ESTATE. */
int cumwin_full(cumwin_t h, int order, double* out_dev);

/* Copy the current moment tensor M_s about the shift vector, i.e. the moments
 * (Eq. 5) of x - shift; the shift is zero in the FP64 form.  Block layout. */
int cumwin_moments(cumwin_t h, int order, double* out_dev);

/* The shift vector (n floats) into shift_host.  Synchronous. */
int cumwin_shift(cumwin_t h, float* shift_host);

/*
 * Norms of the current cumulants.  Synchronises the handle's stream.
 * fro_host[s-1] = ||C_s||_F (the entry-wise 2-norm of the full n^s tensor,
 * Eq. me; ||C_1|| is the Euclidean norm of the mean), s = 1..d.
 * nu_host[s-1] = nu_s = ||C_s|| / ||C_2||^{s/2} (Eq. mef) for s >= 3, NaN for
 * s < 3; ||C_2|| = 0 (a constant window) gives NaN.  Either pointer may be NULL.
 * Returns ENONFINITE if a non-finite sample has entered the window.
 */
int cumwin_norms(cumwin_t h, double* fro_host, double* nu_host);

/* Squared norms ||C_s||_F^2, s = 1..d, as d doubles in device memory (no sync). */
int cumwin_norms_device(cumwin_t h, double* fro2_dev);

/*
 * Entry-wise k-norms of the current cumulants (Eq. me and Algorithm 5 with a
 * general k >= 1): out_host[s-1] = (sum over all n^s entries |C_s[i]|^k)^(1/k),
 * s = 1..d, each stored block weighted by its multiplicity s!/prod r_l!
 * (Section 4.1); k = 2 gives cumwin_norms.  Order 1 is the mean (not the
 * shifted mean of the mixed forms).  The partial sums are added in a fixed
 * order (deterministic).  Synchronises.  Errors: EINVAL (k < 1), ESTATE.
 */
int cumwin_norms_k(cumwin_t h, double k, double* out_host);

/*
 * Univariate diagnostics of the current window (the quantities of Fig. 1 of
 * Section 4.2): per variable i, the skewness C_3[iii] / C_2[ii]^(3/2) and the
 * excess kurtosis C_4[iiii] / C_2[ii]^2 of its marginal, n doubles each (NaN
 * where the order is above d or C_2[ii] = 0).  Either pointer may be NULL.
 * Synchronises.  Errors: EINVAL, ESTATE.
 */
int cumwin_marginals(cumwin_t h, double* skew_host, double* kurt_host);

/* Recompute the moment sums from the window held in the ring buffer (the
 * "simple recalculation" the update is compared against in Section 3.2), then
 * the cumulants and norms. */
int cumwin_recompute(cumwin_t h);

/* Mixed forms: re-fix the shift vector at the current window's column means
 * (FP32-rounded) and recompute the moment sums, the batch-sum FIFO, the
 * cumulants and the norms about it.  The moments are accumulated about that
 * vector, so when the stream's mean has drifted far from the one of the first
 * window, the raw-moment cancellation (and with it the split form's error)
 * grows; this call removes it at the cost of one recomputation.  Cumulants of
 * order >= 2 do not depend on the shift.  In the FP64 form (no shift) it is
 * cumwin_recompute.  Asynchronous; errors: EINVAL, ESTATE. */
int cumwin_recenter(cumwin_t h);

/*
 * Automatic re-centring (mixed forms; not in the paper).  The moments are
 * accumulated about the shift vector fixed at cumwin_fill; when the stream's
 * mean moves away from it, the raw-moment cancellation in the recovery grows
 * (cumwin_recenter).  With limit > 0, every recovery of orders 1-2 measures
 * the drift r = max_i |mean_i - shift_i| / sqrt(C_2[i,i]) on the device and,
 * when r > limit, raises a flag in mapped host memory.  Each eager cumwin_push
 * (not one under stream capture) first waits for the recovery of the push two
 * before it, so that the flag lags the stream by at most two shifts and the
 * host runs at most two shifts ahead of the device; when the flag is up it
 * waits for the pending recoveries and re-centres before its shift.  limit = 0
 * turns it off (the default).  Synchronises.
 * Errors: EINVAL (limit < 0 or not finite, d < 2), ENOTSUP (FP64 form).
 */
int cumwin_set_auto_recenter(cumwin_t h, double limit);

/* The drift ratio r of the last recovery that measured it (NaN before any;
 * measured only while automatic re-centring is on) and the number of
 * automatic re-centrings so far.  Either pointer may be NULL.  Synchronises. */
int cumwin_drift(cumwin_t h, double* ratio_host, int64_t* recenters);

/* Copy the current window, oldest sample first, T x n FP32 row-major (ld = n). */
int cumwin_window(cumwin_t h, float* out_dev);

/*
 * Gradient of L = sum_{s=1..d} w[s] ||C_s||_F^2 (w has d+1 entries, w[0]
 * ignored; full-tensor norms, i.e. each stored block weighted by its
 * multiplicity d!/prod r_l! of Algorithm 5) with respect to the current
 * window, oldest sample first, into dX_dev (T x n FP32, ld = n).  Not in the
 * paper: it is the adjoint of Algorithms 2-4.  The reverse recursion keeps
 * full n^s tensors in FP64 (allocated by the first call; n^d must be at most
 * 2^27, else ENOTSUP); the final contraction with the window runs in FP32.
 * Asynchronous on the handle's stream; w_host is read before returning.
 */
int cumwin_grad(cumwin_t h, const double* w_host, float* dX_dev);

/*
 * Kernel timing.  With timing enabled, each later fill / push / recompute
 * records CUDA events on the handle's stream that split it into staging
 * (X_(+)/X_(-) staging and, in the mixed forms, the operand build), the
 * moment-sum update kernel, and the cumulant recovery + norm kernels (at most
 * 65536 shifts are recorded; later ones are not timed).  cumwin_get_timing
 * synchronises and returns the summed event times in milliseconds, the number
 * of timed shifts and the number of kernels the library launched since timing
 * was enabled.  Enabling resets the counters.  Not for use inside stream capture.
 * enable == 2 records no event between the staging and the update (an event
 * there separates the operand build from the GEMM, which otherwise launch
 * chained); the staging time is then reported inside update_ms and stage_ms
 * is 0.  Timed pushes run their recovery on the handle's stream (no
 * pipelining), so that the three intervals follow each other.
 */
int cumwin_set_timing(cumwin_t h, int enable);
int cumwin_get_timing(cumwin_t h, double* stage_ms, double* update_ms, double* cumulant_ms,
                      int64_t* shifts, int64_t* launches);

/*
 * Autotune the tensor-core update of this handle (mixed forms; not in the
 * paper).  On the data of the last shift it times `reps` launches of the
 * update GEMM for each tile shape -- at most 128 or 64 rows of the left factor
 * per work item, and items issued in super-blocks of 1, 4, 8 or 16 row tiles
 * by all their column tiles, so that the CTAs running together share operand
 * tiles in L2 -- keeps the fastest, then times each split of the samples over
 * CTAs (1, 2, 4, ... up to a workspace limit) and keeps the fewest splits
 * within 10% of the fastest; *ksplit_out receives the split (0 in the FP64
 * form).  When the environment variable CUMWIN_TUNE_CACHE names a file, the
 * choice is appended to it and later handles of the same problem on the same
 * device start from it.  Requires a prior fill; synchronises.
 */
int cumwin_tune(cumwin_t h, int reps, int* ksplit_out);

/* The update's current tile choice: K-split, rows per item, super-block height
 * (all 0 in the FP64 form).  Any pointer may be NULL. */
int cumwin_get_tiles(cumwin_t h, int* ksplit, int* nmax, int* group);
/* Pin a tile choice instead of tuning: ksplit in [1, the plan's limit], nmax a
 * multiple of 16 in [16, 128], group >= 1 (EINVAL otherwise; a no-op in the
 * FP64 form).  At a fixed K-split the results do not depend on the tile shape.
 * Synchronises the device. */
int cumwin_set_tiles(cumwin_t h, int ksplit, int nmax, int group);

/*
 * Batches: many independent windows (streams) of uneven n and d, with a
 * common block size b, shift size p and precision (mixed forms only), advanced
 * together: every phase of a shift (staging, operand build, the tensor-core
 * update, the recovery of each order, the norms) covers all windows, so a
 * shift costs the same number of launches for 1 or 1000 windows -- one when
 * every d <= 4 (cumwin_batch_set_single_launch) -- and can be captured into
 * one CUDA graph.
 */
typedef struct cumwin_batch_s* cumwin_batch_t;

/* Create a batch of nwin windows: window i has n[i] variables, orders 1..d[i],
 * window length T[i].  Errors as for cumwin_create; ENOTSUP for CUMWIN_FP64. */
int cumwin_batch_create(int nwin, const int* n, const int* d, const int64_t* T, int b, int p, int precision,
                        void* cuda_stream, cumwin_batch_t* out);
int cumwin_batch_destroy(cumwin_batch_t B);

/* First windows: X_dev[i] (a host array of nwin device pointers) holds T[i] x n[i]
 * samples of window i, row-major with row stride n[i]. */
int cumwin_batch_fill(cumwin_batch_t B, const float* const* X_dev);

/* Element offset of window i's rows in the packed push buffer (i in [0, nwin];
 * offset(nwin) is the buffer length), -1 on a bad argument. */
int64_t cumwin_batch_offset(cumwin_batch_t B, int window);

/* One shift of every window: x_dev holds, at cumwin_batch_offset(B, i), the p
 * new rows of window i (p x n[i], row-major, row stride n[i]).  Asynchronous;
 * allocates nothing (capturable into a CUDA graph). */
int cumwin_batch_push(cumwin_batch_t B, const float* x_dev);

/* C_s of window i (block layout, as cumwin_cumulants). */
int cumwin_batch_cumulants(cumwin_batch_t B, int window, int order, double* out_dev);

/* Norms of all windows: fro_host and nu_host are nwin x dmax (dmax = the
 * largest d), row i for window i, NaN beyond d[i] (and for nu below order 3).
 * Synchronises; returns ENONFINITE / ETIMEOUT if any window saw one. */
int cumwin_batch_norms(cumwin_batch_t B, double* fro_host, double* nu_host);

/* Autotune the batch's update GEMM (as cumwin_tune), and its tile choice. */
int cumwin_batch_tune(cumwin_batch_t B, int reps, int* ksplit_out);
int cumwin_batch_get_tiles(cumwin_batch_t B, int* ksplit, int* nmax, int* group);

/* 1 when the batch's shifts use the batch-sum FIFO (every T[i] a multiple of
 * p and room for it, see cumwin_push), 0 otherwise, EINVAL. */
int cumwin_batch_fifo(cumwin_batch_t B);

/*
 * Single-launch shifts (not in the paper).  When every window's orders are
 * recovered by the fused recovery (d <= 4) and the device can keep one
 * 1024-thread CTA with the GEMM's shared memory on every SM, cumwin_batch_push
 * runs a whole shift -- staging, operand build, the tensor-core update and the
 * recovery of every order with the norms -- as one cooperative launch whose
 * phases are separated by bounded grid barriers (on by default).  enable = 0
 * runs the phases as separate launches instead; the results are the same.
 * Returns 1 when single-launch shifts are available for this batch, 0 when not,
 * EINVAL for a null handle.
 */
int cumwin_batch_set_single_launch(cumwin_batch_t B, int enable);

/* Kernels launched by the last cumwin_batch_push (staging, operand build,
 * GEMM and the recovery's launches; 1 for a single-launch shift); 0 before the
 * first push, EINVAL for a null handle.  Host bookkeeping only: it does not
 * synchronise. */
int64_t cumwin_batch_launches(cumwin_batch_t B);

/* Sticky device status over all windows (synchronises). */
int cumwin_batch_status(cumwin_batch_t B);

/* Sticky device status of the handle (CUMWIN_OK or ENONFINITE / ETIMEOUT).
 * Synchronises the handle's stream.  Reading it clears nothing. */
int cumwin_status(cumwin_t h);

/*
 * Allocation-free squared norm of a tensor in the block layout.  The paper has
 * no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc, such as code running inside another framework's memory pool or
 * under a device-memory budget that forbids new allocations, or a thread that
 * must not risk the implicit synchronisation an allocation can bring.
 *
 * out_dev[0] = sum over stored blocks j of (order!/prod r_l!) * sum_{e in block j} e^2,
 * where r_l are the run lengths of equal entries of the sorted block index j,
 * i.e. ||A||_F^2 of the full n^order tensor, for A_dev in the block layout
 * (cumwin_layout_size(n, b, order) doubles, device).  Asynchronous on
 * cuda_stream; the caller passes the input and the output and the call
 * allocates nothing: its scratch, one double per stored block, is a fixed
 * array of CUMWIN_NOALLOC_MAX_BLOCKS doubles in the library's device memory,
 * which every GPU that loads the library holds until the process exits.
 * Errors (returned before anything is launched): EINVAL for a bad argument,
 * for ceil(n/b)*b > CUMWIN_MAX_N or b^order >= 2^31, and for tensors with more
 * stored blocks than the scratch holds (with a message in cumwin_last_error());
 * ECUDA for a failed CUDA call.
 * The scratch's device address is looked up (with the current device) on
 * every call made outside stream capture, so a device reset does not leave a
 * stale address; a call made while cuda_stream is being captured reuses the
 * address of the last uncaptured call on that device, so the first call on a
 * device must come before any stream capture (ESTATE otherwise).  All calls
 * share the one scratch array and each call overwrites the slots it reads, so
 * calls that overlap on the GPU (different streams without ordering) race and
 * may return wrong sums.
 */
#define CUMWIN_NOALLOC_MAX_BLOCKS 16384
int cumwin_block_norm2_noalloc(int n, int b, int order, const double* A_dev, double* out_dev,
                               void* cuda_stream);

/* Host-only layout helpers (no GPU needed). */
/* Stored elements of order `order`: C(nbar + order - 1, order) * b^order. */
int64_t cumwin_layout_size(int n, int b, int order);
/* Lexicographic rank of the sorted block multi-index j (order entries,
 * 0 <= j[0] <= ... < nbar); -1 if j is not sorted or out of range. */
int64_t cumwin_block_rank(int n, int b, int order, const int* j);
/* Storage index of the tensor entry at variable multi-index i (any order of
 * its entries, each in [0, n)); -1 on a bad argument. */
int64_t cumwin_element_index(int n, int b, int order, const int* i);
/* Self-test of the host tables that map update tiles and cumulant sub-blocks
 * to storage indices against a direct enumeration (0 = pass): the full update
 * tables, the canonical-element tables, the compressed update tables (every
 * canonical element produced once, at the workspace slot its rank pair gives)
 * and the sub-block lookups of the recovery; a positive code names the first
 * check that failed. */
int cumwin_selftest_tables(int n, int b, int order);

/* Message for a return code, and the detail of the last CUDA error seen by
 * the calling thread. */
const char* cumwin_strerror(int code);
const char* cumwin_last_error(void);

/* Library version, e.g. 100 for 0.1.0. */
int cumwin_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CUMWIN_H */
