/*
 * kkm.h -- C ABI of a GB300 (sm_103a) library for approximate mini-batch
 * kernel k-means (Ferrarotti, Decherchi & Rocchia, "Distributed kernel
 * k-means for large scale clustering", arXiv 1710.03013).
 *
 * Conventions shared by every call
 *   - Matrices are row-major float32.  A "sample" is one row of length d.  For
 *     the molecular-dynamics kernel (KKM_RMSD) a row holds one frame as
 *     [n_atoms][3] coordinates, so d == 3 * n_atoms.
 *   - Input pointers may point to device memory (e.g. a CUDA tensor) or to
 *     host memory; the library detects which with cudaPointerGetAttributes and
 *     copies host inputs to the device itself.  Output pointers follow the
 *     same rule unless the comment says "host".
 *   - The caller owns every buffer it passes and keeps it valid until the call
 *     returns.  Calls run in stream order on the given stream (NULL = the
 *     legacy default stream) and are synchronous: results are complete when
 *     the call returns.
 *   - No call aborts, traps or throws.  Errors are returned as kkm_status; a
 *     readable message for the calling thread is in kkm_last_error().  Invalid
 *     arguments give KKM_EINVAL and write nothing.
 *   - Work is deterministic: the same inputs, seed and options give
 *     bit-identical results.
 */
#ifndef KKM_H
#define KKM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum kkm_status {
  KKM_OK = 0,
  KKM_EINVAL = 1,    /* invalid argument (sizes, NaN/Inf inputs, bad kernel) */
  KKM_ENOMEM = 2,    /* device allocation failed                            */
  KKM_EBUDGET = 3,   /* refused by a memory budget                          */
  KKM_ECUDA = 4,     /* a CUDA runtime call failed                          */
  KKM_ETIMEOUT = 5,  /* a bounded device wait gave up                       */
  KKM_EINTERNAL = 6  /* internal inconsistency                              */
} kkm_status;

/* Kernel functions (Section 2 replaces feature-space products by a Mercer
 * kernel K; the paper uses a Gaussian kernel and, for MD frames, asks for
 * roto-translational invariance without writing the kernel down):
 *   KKM_RBF    K(x,y) = exp(-||x-y||^2 / (2 sigma^2))
 *   KKM_RMSD   K(x,y) = exp(-rmsd(x,y)^2 / (2 sigma^2)), rmsd after optimal
 *              proper superposition of the mean-centred frames (QCP root)
 *   KKM_LINEAR K(x,y) = x . y  (kernel k-means then equals Lloyd k-means)   */
typedef enum kkm_kernel_kind { KKM_RBF = 0, KKM_RMSD = 1, KKM_LINEAR = 2 } kkm_kernel_kind;

/* Arithmetic of the kernel-block evaluation K(X^i, L).  KKM_FP32 is the
 * plain FFMA path.  KKM_BF16 (RBF and linear kernels) runs the Gram product
 * on the tensor cores from BF16-rounded rows with FP32 accumulation; the
 * C-column blocks (Eq. 8, 12, k-means++) and all sums stay FP32/FP64.
 * KKM_FP8 (RBF and linear kernels) runs it on e4m3 rows, each scaled by
 * max |x| / 448 (tcgen05 kind::f8f6f4, FP32 accumulation).  Both store the
 * Gaussian block in FP16 and re-score near-tie rows from FP32 kernel values
 * (the window is 1e-3 of the term scale for BF16, 3e-2 for FP8).  Rows of at
 * most 128 values use the FP32 Gram stored in FP16 on both. */
typedef enum kkm_precision { KKM_FP32 = 0, KKM_BF16 = 1, KKM_FP8 = 2 } kkm_precision;

/* Mini-batch fetching (Section 3.1): stride X^i = {x_(i+jB)}; block = B
 * contiguous pieces, the first N mod B one sample longer.                   */
typedef enum kkm_sampling { KKM_STRIDE = 0, KKM_BLOCK = 1 } kkm_sampling;

/* Scheduling of the kernel blocks (Section 4, Fig. 3: the block of the next
 * mini-batch is produced while the current one iterates).  KKM_PIPE_OVERLAP
 * computes K(X^(i+1), L^(i+1)) on a low-priority stream while mini-batch i
 * runs its inner loop on a high-priority one (two block buffers);
 * KKM_PIPE_SERIAL computes each block just before its inner loop (one
 * buffer).  KKM_PIPE_AUTO overlaps when B >= 2 except for a reduced-precision
 * RBF/linear block streamed by the split loop (a few percent of such a fit,
 * whose writes would evict the cached block the loop streams); with the
 * tensor-core loop (KKM_ITER_TC) the next block runs on the SMs the loop
 * leaves free.  In kkm_fit_batch and the server,
 * whose fits already run side by side, AUTO means serial.  The results are
 * the same bits either way: the same kernels run on the same inputs.       */
typedef enum kkm_pipeline { KKM_PIPE_AUTO = 0, KKM_PIPE_SERIAL = 1, KKM_PIPE_OVERLAP = 2 } kkm_pipeline;

/* Launch form of the inner loop (Eq. 15-17).  KKM_ITER_FUSED runs all the
 * iterations of a mini-batch in one cooperative launch: every CTA owns a
 * strip of sample columns over all landmark rows, so f_hat is finished where
 * it is summed, and grid barriers make g_hat (Eq. 16) and the cost available
 * to every CTA.  It applies to C <= 64 and mini-batches of up to about
 * 77,000 samples (KKM_EINVAL otherwise).
 * KKM_ITER_TC is the same one-launch loop with the f_hat sums formed on the
 * tensor cores, as the product of the FP16-stored Gaussian block with the
 * one-hot matrix of the landmark labels (exact 0/1 values, FP32
 * accumulation): one CTA per 128 samples.  It applies to the RBF kernel with
 * KKM_BF16 or KKM_FP8, C <= 16 and mini-batches of at most 128 samples per SM
 * (19,456 on 152 SMs) whose landmark one-hot tiles fit in shared memory
 * (about 3,000 landmarks) (KKM_EINVAL otherwise).
 * KKM_ITER_SPLIT streams per-unit partial sums and finishes them in a second
 * launch (the two launches of an iteration chained by programmatic
 * dependent launch).  KKM_ITER_AUTO takes KKM_ITER_TC where it applies and
 * the split form elsewhere.  Fits that run side by side (kkm_fit_batch,
 * kkm_fit_restarts, kkm_elbow, the server) take the split form whatever the
 * option: the one-launch forms wait at grid barriers for all their CTAs,
 * which other fits' one-launch loops could hold off.  The forms add the same
 * values in different orders: labels agree above the tolerance margin and
 * distances to FP32 rounding.                                               */
typedef enum kkm_iteration {
  KKM_ITER_AUTO = 0,
  KKM_ITER_FUSED = 1,
  KKM_ITER_SPLIT = 2,
  KKM_ITER_TC = 3
} kkm_iteration;

/* Prototypes used by kkm_assign / kkm_cost: the sparse landmark centroids
 * of the last mini-batch (Eq. 14-17) or the global medoids (Eq. 2 against
 * the output M of Algorithm 1).                                             */
typedef enum kkm_assign_mode { KKM_ASSIGN_SUPPORTS = 0, KKM_ASSIGN_MEDOIDS = 1 } kkm_assign_mode;

typedef struct kkm_kernel {
  int32_t kind;     /* kkm_kernel_kind                                         */
  float sigma;      /* Gaussian width; <= 0 asks kkm_fit for the median rule   */
  int32_t n_atoms;  /* KKM_RMSD only: atoms per frame (d == 3 * n_atoms)       */
} kkm_kernel;

typedef struct kkm_options {
  int32_t precision;            /* kkm_precision (default KKM_FP32)             */
  int32_t sampling;             /* kkm_sampling (default KKM_STRIDE)            */
  int32_t early_stop;           /* 1: stop an inner loop when no label changes */
  int32_t pipeline;             /* kkm_pipeline (default KKM_PIPE_AUTO)         */
  int32_t iteration;            /* kkm_iteration (default KKM_ITER_AUTO)        */
  const int64_t* init_medoids;  /* host [C] global sample indices replacing
                                   kernel k-means++, or NULL                    */
  void* stream;                 /* cudaStream_t or NULL                         */
} kkm_options;

/* A fitted model.  It owns device copies of everything it keeps (medoid and
 * landmark coordinates, landmark labels, compactness g_hat); nothing aliases
 * the caller's data.                                                        */
typedef struct kkm_model kkm_model;

/* Fills *opt with the defaults listed above (early_stop = 1). */
void kkm_options_default(kkm_options* opt);

/*
 * kkm_fit -- Algorithm 1 with the landmark approximation of Section 3.2.
 *   X        [N][d] float32 samples (device or host).  Device and pageable
 *            host X are checked for NaN/Inf before any other work (host X is
 *            copied first).  Pinned host X (16-byte aligned, d a multiple of
 *            4, RBF or linear kernel) stays on the host: each mini-batch's
 *            rows are fetched by the copy engine as the fit reaches them (the
 *            next mini-batch's while the current one iterates) and checked
 *            there; a NaN/Inf then gives KKM_EINVAL at the end of the fit with
 *            no label or model written.  The host memory must stay unchanged
 *            until the call returns.
 *   C        number of clusters, 1 <= C <= 256 and C <= every mini-batch size.
 *   B        number of mini-batches, 1 <= B <= N.
 *   s        landmark fraction of Eq. 18, 0 < s <= 1; per mini-batch
 *            |L| = clamp(ceil(s N_i - 1e-9), 1, N_i), computed in double.
 *   k        kernel; sigma <= 0 selects the median pairwise distance of up to
 *            2048 samples drawn with the seed (not allowed for KKM_LINEAR).
 *   iters    cap on inner iterations per mini-batch (>= 0).
 *   seed     seeds SplitMix64; its draws seed k-means++, the bandwidth sample
 *            and one landmark draw per mini-batch, in that order.
 *   opt      options or NULL for the defaults.
 *   labels_out [N] int32 (device or host, nullable): each sample's final
 *            label in its own mini-batch.
 *   model_out  receives a new model (free with kkm_model_free), nullable.
 * Per mini-batch it evaluates the block K(X^i, L) once (Alg. 1 line 3),
 * initialises labels from the global medoids (Eq. 8, k-means++ on the first
 * mini-batch), iterates Eq. 15-17, then computes the mini-batch medoids
 * (Eq. 10) and merges them into the global ones (Eq. 11-13).
 * Errors: KKM_EINVAL for bad sizes, s outside (0,1], d != 3 n_atoms, C larger
 * than a mini-batch, non-finite X or out-of-range init_medoids.
 */
kkm_status kkm_fit(const float* X, int64_t N, int64_t d, int32_t C, int32_t B,
                   double s, const kkm_kernel* k, int32_t iters, uint64_t seed,
                   const kkm_options* opt, int32_t* labels_out,
                   kkm_model** model_out);

/* The state of a fit between two mini-batches: what Algorithm 1 carries from
 * one outer iteration to the next (the global medoids and their cumulative
 * counts of Eq. 11-13), the bandwidth in use, the trace and the centre
 * displacements so far, and the arguments of the fit that made it.  Host
 * memory only; nothing on the device.                                       */
typedef struct kkm_checkpoint kkm_checkpoint;

/*
 * kkm_fit_range -- kkm_fit over the mini-batches [start, stop) only, so that a
 * long fit can be stopped after any mini-batch and resumed later, in this
 * process or another one.  The paper runs Algorithm 1 in one pass; this is a
 * library service around its outer loop.
 *   from     NULL: start = 0 (k-means++ or init_medoids, the bandwidth rule);
 *            else a checkpoint of an earlier call with the same X (same rows
 *            in the same order), N, d, C, B, s, kernel, iters, seed and
 *            opt.precision / sampling / early_stop / init_medoids (given or
 *            not); start = its next mini-batch.  Other arguments give
 *            KKM_EINVAL.  opt.pipeline, opt.iteration and opt.stream may
 *            differ between calls.
 *   stop     one past the last mini-batch of this call, start < stop <= B.
 *   labels_out [N] int32 (device or host, nullable): the labels of the rows
 *            of mini-batches [start, stop); other rows keep their values.
 *   model_out  nullable; only with stop == B (else KKM_EINVAL).
 *   ckpt_out   nullable; receives a new checkpoint after mini-batch stop - 1
 *            (free with kkm_checkpoint_free).
 * Calls over [0, b1), [b1, b2), ..., [bk, B) chained through their
 * checkpoints give the labels, model, trace and displacements of one kkm_fit
 * call with the same arguments, bit for bit.  Errors as kkm_fit.
 */
kkm_status kkm_fit_range(const float* X, int64_t N, int64_t d, int32_t C,
                         int32_t B, double s, const kkm_kernel* k,
                         int32_t iters, uint64_t seed, const kkm_options* opt,
                         const kkm_checkpoint* from, int32_t stop,
                         int32_t* labels_out, kkm_model** model_out,
                         kkm_checkpoint** ckpt_out);

/* kkm_checkpoint_info -- the next mini-batch, B, C and the bandwidth of a
 * checkpoint; medoids_out [C] int64 (host, nullable) gets the global medoids
 * (sample indices) after mini-batch next_batch - 1.  Outputs are nullable. */
kkm_status kkm_checkpoint_info(const kkm_checkpoint* c, int32_t* next_batch,
                               int32_t* B, int32_t* C, float* sigma,
                               int64_t* medoids_out);

/* kkm_checkpoint_save / kkm_checkpoint_load -- a checkpoint to and from a
 * little-endian file with the magic "KKMCKP01".  Loading checks every field
 * (sizes, ranges, the file length) and gives KKM_EINVAL for a file that is
 * not a consistent checkpoint.  Host only; synchronous. */
kkm_status kkm_checkpoint_save(const kkm_checkpoint* c, const char* path);
kkm_status kkm_checkpoint_load(const char* path, kkm_checkpoint** out);
void kkm_checkpoint_free(kkm_checkpoint* c);

/* One problem of a batched fit: the arguments of one kkm_fit call. */
typedef struct kkm_problem {
  const float* X;       /* [N][d] device or host                            */
  int64_t N, d;
  int32_t C, B;
  double s;
  kkm_kernel kernel;
  int32_t iters;
  uint64_t seed;
  kkm_options opt;      /* opt.stream is ignored (the batch uses its own)   */
  int32_t* labels_out;  /* [N] device or host, nullable                     */
} kkm_problem;

/*
 * kkm_fit_restarts -- Section 4.5: the method initialised several times with
 * kernel k-means++ and the solution of minimum cost kept.  Restart r is
 * kkm_fit with the r-th output of SplitMix64(seed) as its seed; all restarts
 * run as one kkm_fit_batch.  With sigma <= 0 the median rule is applied once
 * (kkm_median_bandwidth with `seed`) and every restart uses that bandwidth,
 * so that their costs compare fits of one kernel.  The cost of a restart is
 * Eq. 1 over X against its final global medoids (kkm_cost with
 * KKM_ASSIGN_MEDOIDS); the lowest cost wins, ties to the lowest restart.
 *   n_restarts 1..1024; opt as for kkm_fit (init_medoids must be NULL).
 *   labels_out [N] (device or host, nullable), model_out (nullable): the
 *   winner's labels and model.  costs_out [n_restarts] (host, nullable),
 *   best_out (host, nullable): every restart's cost and the winner's index.
 */
kkm_status kkm_fit_restarts(const float* X, int64_t N, int64_t d, int32_t C,
                            int32_t B, double s, const kkm_kernel* k,
                            int32_t iters, uint64_t seed, int32_t n_restarts,
                            const kkm_options* opt, int32_t* labels_out,
                            kkm_model** model_out, double* costs_out,
                            int32_t* best_out);

/*
 * kkm_elbow -- the number of clusters by the elbow criterion (Sections 4.4
 * and 4.5 choose C this way over a range, (4, 40) for the MD trajectory).
 * For every C in [C_lo, C_hi] the best of n_restarts restarts (the rule and
 * seeds of kkm_fit_restarts, the same seeds for every C); all (C, restart)
 * fits run as one kkm_fit_batch.  The paper does not define the criterion;
 * the C returned is the one whose cost lies farthest below the chord joining
 * the end points of the cost curve, both axes scaled to [0, 1] (lowest C on
 * ties).  1 <= C_lo < C_hi <= 256.  costs_out [C_hi - C_lo + 1] (host,
 * nullable) gets each C's minimum cost; *C_out (host) the elbow.
 */
kkm_status kkm_elbow(const float* X, int64_t N, int64_t d, int32_t C_lo,
                     int32_t C_hi, int32_t B, double s, const kkm_kernel* k,
                     int32_t iters, uint64_t seed, int32_t n_restarts,
                     const kkm_options* opt, double* costs_out, int32_t* C_out);

/*
 * kkm_fit_batch -- n independent fits on one GPU at once: many data sets of
 * uneven sizes, or restarts of one data set with different seeds.  Each
 * problem gets exactly the results of kkm_fit with the same arguments and
 * opt.iteration = KKM_ITER_SPLIT (the loop form of fits side by side).  The
 * paper fits one data set at a time; this is a library service around
 * Algorithm 1, not a change to it.
 *   problems   [n] host array.
 *   n_streams  concurrent fits (one host worker thread and CUDA stream
 *              each), 1..64, or 0 for the default (32).  Fits start longest
 *              first.  Their inner loops run as work lists: one launch per
 *              step of an iteration covers every loop in flight (each loop's
 *              CTAs compute what its own launches would), on a stream of the
 *              call's own.  The rows per CTA of those assign launches (1, 2,
 *              4 or 8 blocks of 32; no effect on results) are chosen by
 *              timing per launch size and kept for the process; the
 *              environment variable KKM_TUNE_CACHE names a file that keeps
 *              the choices across processes, KKM_ASSIGN_ROWS forces one.
 *              KKM_LOOP_CHAINS (1..8) sets how many such work-list streams
 *              the call runs side by side (each fit's loops go to one of
 *              them; no effect on results).
 *   models_out [n] host array of model pointers (nullable); a failed
 *              problem's entry is NULL.
 *   status_out [n] host array: each problem's status.
 *   stream     work queued on this stream before the call (e.g. the copies
 *              that produced the inputs) completes before any fit starts.
 * Returns KKM_OK when every problem succeeded, else the status of the
 * lowest-numbered failing problem (kkm_last_error names it); the other
 * problems still run to completion.  Synchronous: returns when all are done.
 */
kkm_status kkm_fit_batch(const kkm_problem* problems, int32_t n, int32_t n_streams,
                         kkm_model** models_out, kkm_status* status_out, void* stream);

/*
 * Serving: a request loop for fit and assign jobs on one GPU.  The paper has
 * no serving layer; this is a library service around Algorithm 1 (fits) and
 * Eq. 15 (assignment of new samples to resident models).
 *
 * Jobs are queued by kkm_server_submit_* from any host thread and run on
 * worker threads, each with its own CUDA stream, as soon as a worker is free
 * and the job's device-memory estimate fits in the budget beside the
 * resident models and the running jobs; so jobs that arrive while others run
 * overlap on the device.  Waiting assign jobs on the same model and mode are
 * fused into one launch; each row's result is bit-for-bit what the request
 * would get alone.  Later jobs may pass one that does not fit yet, at most
 * 16 times.  Buffers passed to a submit call (host or device) must stay
 * valid until kkm_server_wait reports the job finished.
 */
typedef struct kkm_server kkm_server;

typedef struct kkm_server_config {
  uint64_t budget_bytes;   /* HBM admission budget (resident models + running jobs) */
  int32_t n_workers;       /* concurrent jobs (one stream each); 0: 4, at most 64   */
  int32_t reserved;        /* must be 0                                             */
  int64_t max_batch_rows;  /* rows of fused assign jobs per launch; 0: 65536        */
} kkm_server_config;

typedef struct kkm_serving_stats {
  int64_t completed_fit, completed_assign, failed, refused;
  int64_t fused_assign_launches;  /* kkm_assign launches that served the assign jobs */
  int64_t queued;                 /* jobs waiting for admission now                  */
  double p50_fit_ms, p99_fit_ms;  /* submit-to-finish latency of completed jobs       */
  double p50_assign_ms, p99_assign_ms;
  double kernel_evals;            /* kernel evaluations of the completed jobs         */
  double seconds;                 /* since creation or the last kkm_server_reset_stats */
  uint64_t bytes_in_use, peak_bytes;  /* admission accounting (estimates)            */
} kkm_serving_stats;

/* Starts the workers.  KKM_EINVAL for a zero budget or n_workers > 64. */
kkm_status kkm_server_create(const kkm_server_config* cfg, kkm_server** out);
/* Runs every queued job to the end, stops the workers, frees the resident
 * models and the server. */
void kkm_server_destroy(kkm_server* s);
/* Makes a fitted model resident; the server takes ownership (do not free it).
 * KKM_EBUDGET if the resident models would exceed the budget. */
kkm_status kkm_server_add_model(kkm_server* s, kkm_model* m, int32_t* model_id);
/* Releases a resident model (after its running jobs); KKM_EINVAL if jobs
 * for it are still queued or the id is unknown. */
kkm_status kkm_server_remove_model(kkm_server* s, int32_t model_id);
/* Queues kkm_fit(p...) (p->opt.stream is ignored).  keep_model != 0 makes the
 * fitted model resident; kkm_server_wait then gives its id.  KKM_EBUDGET if
 * the job could never fit in the budget. */
kkm_status kkm_server_submit_fit(kkm_server* s, const kkm_problem* p, int32_t keep_model,
                                 uint64_t* ticket);
/* Queues kkm_assign(model, X[M][d], mode) into labels_out[M] and dist_out[M]
 * (nullable), host or device memory. */
kkm_status kkm_server_submit_assign(kkm_server* s, int32_t model_id, const float* X, int64_t M,
                                    int32_t mode, int32_t* labels_out, float* dist_out,
                                    uint64_t* ticket);
/* Waits up to timeout_ms (< 0: no limit) for the job.  On KKM_OK the job has
 * finished: *job_status is its status (kkm_last_error has its message) and
 * *model_id_out (nullable) the id of a kept model, else -1; the ticket is
 * then consumed.  KKM_ETIMEOUT if it has not finished in time. */
kkm_status kkm_server_wait(kkm_server* s, uint64_t ticket, int32_t timeout_ms,
                           kkm_status* job_status, int32_t* model_id_out);
kkm_status kkm_server_stats(kkm_server* s, kkm_serving_stats* out);
kkm_status kkm_server_reset_stats(kkm_server* s);

/*
 * kkm_assign -- label new samples against a fitted model: Eq. 15 with the
 * model's landmark supports (mode KKM_ASSIGN_SUPPORTS) or Eq. 2 against its
 * medoids (KKM_ASSIGN_MEDOIDS).  Ties go to the lowest cluster index.
 *   Xnew [M][d] float32, labels_out [M] int32, dist_out [M] float32 squared
 *   feature-space distance to the chosen prototype (nullable).  M may be 0.
 */
kkm_status kkm_assign(const kkm_model* m, const float* Xnew, int64_t M,
                      int32_t mode, int32_t* labels_out, float* dist_out,
                      void* stream);

/* kkm_cost -- Eq. 1 for samples X against the model's prototypes:
 * *omega_out (host) = sum_i min_j ||phi(x_i) - w_j||^2, accumulated in FP64. */
kkm_status kkm_cost(const kkm_model* m, const float* X, int64_t N, int32_t mode,
                    double* omega_out, void* stream);

/* Model accessors.  All outputs are host memory unless stated. */
kkm_status kkm_model_info(const kkm_model* m, int32_t* C, int64_t* d,
                          int32_t* n_support, float* sigma);
/* idx_out [C] global sample indices of the medoids; counts_out [C] the
 * cumulative member counts |w_j| of Eq. 13 (nullable); coords_out [C][d]
 * medoid coordinates (device or host, nullable). */
kkm_status kkm_model_medoids(const kkm_model* m, int64_t* idx_out,
                             int64_t* counts_out, float* coords_out);
/* Final supports of the last mini-batch: landmark labels [n_support],
 * g_hat [C] (Eq. 16) and landmark counts n_j [C]; each nullable. */
kkm_status kkm_model_supports(const kkm_model* m, int32_t* labels_out,
                              double* ghat_out, int32_t* n_out);
/* Average displacement of the cluster centres in each outer iteration
 * (Section 4.1, Fig. 4b, proposed there as the observable of sampling
 * quality): for mini-batch i, the mean over the C clusters of the
 * feature-space distance sqrt(K(a,a) - 2K(a,b) + K(b,b)) between the global
 * medoid a before and b after the mini-batch (0 for an unchanged medoid).
 * Up to cap values to out (host, nullable); *n_out gets B. */
kkm_status kkm_model_displacement(const kkm_model* m, double* out, int32_t cap,
                                  int32_t* n_out);
/* Inner-loop trace over all mini-batches: Omega (Eq. 9) and the number of
 * changed labels of each executed iteration, up to cap entries; *n_out gets
 * the total number of entries. */
kkm_status kkm_model_trace(const kkm_model* m, double* omega, int32_t* changed,
                           int32_t cap, int32_t* n_out);
void kkm_model_free(kkm_model* m);

/* kkm_model_save / kkm_model_load -- a fitted model to and from a file (a
 * little-endian binary with a versioned header), e.g. to restart a serving
 * process without refitting.  The paper has no persistence; this is a
 * library service.  Synchronous.  kkm_model_load allocates the model on the
 * current device; a file that is not a model, or whose header and length
 * disagree, gives KKM_EINVAL before any device work. */
kkm_status kkm_model_save(const kkm_model* m, const char* path);
kkm_status kkm_model_load(const char* path, kkm_model** model_out);

/* kkm_kernel_matrix -- out[a][b] = K(A_a, B_b) for A [nA][d], B [nB][d]
 * (the kernel-block evaluation of Alg. 1 line 3 as a standalone call).
 * out is [nA][nB] float32, device or host.  sigma must be > 0.
 * precision KKM_BF16 (RBF and linear kernels) evaluates the product on the
 * tensor cores from BF16-rounded rows with FP32 accumulation; the result is
 * then the kernel of the rounded rows. */
kkm_status kkm_kernel_matrix(const float* A, int64_t nA, const float* Bm,
                             int64_t nB, int64_t d, const kkm_kernel* k,
                             int32_t precision, float* out, void* stream);

/* kkm_median_bandwidth -- the bandwidth rule kkm_fit applies when sigma <= 0:
 * the lower median of the pairwise distances (Euclidean, or RMSD for
 * KKM_RMSD) among min(N, 2048) samples drawn by the bandwidth stream of
 * `seed`.  *sigma_out is host memory. */
kkm_status kkm_median_bandwidth(const float* X, int64_t N, int64_t d,
                                const kkm_kernel* k, uint64_t seed,
                                float* sigma_out);

/*
 * kkm_debug_step -- one inner iteration (Eq. 15-17) on one mini-batch with
 * the labels given (teacher forcing), for step-by-step checks.
 *   Xb [Ni][d] mini-batch samples; L [nL] sorted local landmark indices
 *   (host); u_in [Ni] labels (host); precision KKM_FP32 or KKM_BF16 (the
 *   kernel block kkm_fit evaluates and stores for that precision, and on
 *   KKM_BF16 its FP32 near-tie re-score); iteration a kkm_iteration (the
 *   launch form of the step).  Outputs (host, each nullable):
 *   u_out [Ni], fhat_out [Ni][C] (Eq. 17 from the stored block, before any
 *   re-score; NaN where n_j = 0), margin_out [Ni] (second-best minus best
 *   distance), ghat_out [C] (Eq. 16; NaN where n_j = 0), n_out [C],
 *   *omega_out, *changed_out.
 */
kkm_status kkm_debug_step(const float* Xb, int64_t Ni, int64_t d,
                          const int32_t* L, int32_t nL, const kkm_kernel* k,
                          int32_t C, int32_t precision, int32_t iteration,
                          const int32_t* u_in, int32_t* u_out,
                          float* fhat_out, float* margin_out, double* ghat_out,
                          int32_t* n_out, double* omega_out,
                          int32_t* changed_out, void* stream);

/* kkm_debug_kmeanspp -- the kernel k-means++ picks kkm_fit makes on its first
 * mini-batch X0 [N0][d] for `seed`: picks_out [C] local indices (host). */
kkm_status kkm_debug_kmeanspp(const float* X0, int64_t N0, int64_t d,
                              const kkm_kernel* k, int32_t C, uint64_t seed,
                              int64_t* picks_out, void* stream);

/* kkm_minibatch_plan -- host-only (no GPU needed): the mini-batch geometry
 * and landmark draw kkm_fit uses for mini-batch `batch` of N samples.
 * Mini-batch `batch` holds the global samples start + l*step, l < *n_out
 * (Section 3.1 sampling); L_out (nullable, capacity *n_out) receives its
 * sorted local landmark indices (Eq. 14, |L| from Eq. 18) and *nl_out their
 * number.  All pointers are host memory. */
kkm_status kkm_minibatch_plan(int64_t N, int32_t B, int32_t sampling, double s,
                              uint64_t seed, int32_t batch, int64_t* start_out,
                              int64_t* step_out, int64_t* n_out, int32_t* L_out,
                              int64_t* nl_out);

/* kkm_assign_noalloc -- kkm_assign for callers that cannot allocate device
 * memory: a request path where cudaMalloc could synchronise the device and
 * stall other work, or a process whose device memory belongs to another
 * framework's pool.  The paper has no counterpart; this is a library service.
 *   Labels and squared distances as kkm_assign computes them, for one chunk
 *   of at most KKM_NOALLOC_MAX_ROWS query rows.  RBF and linear models run
 *   the same kernels as kkm_assign and give the same bits; for an RMSD model
 *   kkm_assign may take its tensor-core screen (32 or more reference rows,
 *   sigma >= 0.5) while this call evaluates every pair exactly, so distances
 *   agree within 1e-5 of the term scale and labels wherever the relative
 *   margin between the two nearest clusters exceeds 1e-4.  The model may
 *   have at most KKM_NOALLOC_MAX_REF reference rows (landmark supports in
 *   mode KKM_ASSIGN_SUPPORTS, medoids in mode KKM_ASSIGN_MEDOIDS) and a
 *   prepared row length of at most KKM_NOALLOC_MAX_ROWLEN floats (d rounded up to 8;
 *   for KKM_RMSD 3 * n_atoms rounded up to 24).  Larger sizes give KKM_EINVAL.
 *   Xnew, labels_out and dist_out (nullable) must be memory of the model's
 *   device, and that device must be current; otherwise KKM_EINVAL.  The call
 *   returns when its work is done: it waits for the stream once after the
 *   non-finite-input check and once at the end.
 * It allocates nothing: its working memory is one fixed scratch array of
 * about 21 MB that every GPU loading this library keeps until exit.  The
 * first call on each device looks up that array's device address (and may
 * load the library's device code); make it before any stream capture.  All
 * calls share the array: calls whose GPU work overlaps (several streams or
 * threads at once) race; calls in order on one stream are safe. */
#define KKM_NOALLOC_MAX_ROWS 1024
#define KKM_NOALLOC_MAX_REF 4096
#define KKM_NOALLOC_MAX_ROWLEN 1024
kkm_status kkm_assign_noalloc(const kkm_model* m, const float* Xnew, int64_t M,
                              int32_t mode, int32_t* labels_out,
                              float* dist_out, void* stream);

const char* kkm_status_string(kkm_status s);
/* Message of the last failed call on this thread ("" if none). */
const char* kkm_last_error(void);

/* Per-kernel device timing.  kkm_prof_enable(1): every library kernel launch
 * is counted and bracketed by CUDA events on its stream; (2): every launch is
 * counted, only the kernel-block and streaming kernels ("gram_block",
 * "rmsd_block", "rmsd_exact", "fhat_partial", "iterate") are bracketed; (0): off.
 * kkm_prof_read returns the number of launches and the summed device
 * milliseconds of the named kernel since the last reset (0 launches if
 * unknown).  kkm_prof_work returns the work units a data-dependent kernel
 * reported while profiling was on ("rmsd_exact": frame pairs recomputed; the
 * count costs a device read-back per launch).  kkm_prof_names writes a
 * comma-separated list of the names seen into buf. */
void kkm_prof_enable(int32_t on);
void kkm_prof_reset(void);
int32_t kkm_prof_read(const char* name, int64_t* launches, double* ms);
double kkm_prof_work(const char* name);
int32_t kkm_prof_names(char* buf, int32_t cap);

#ifdef __cplusplus
}
#endif

#endif /* KKM_H */
