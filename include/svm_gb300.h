/*
 * svm_gb300.h -- C ABI of a GB300-native (sm_103a) kernel-SVM trainer.
 *
 * The library trains a two-class soft-margin SVM with an RBF kernel by the
 * SMO method of "Fast Support Vector Machines Using Parallel Adaptive
 * Shrinking on Distributed Systems" (arXiv:1406.5161):
 *   - the dual problem of Section II-A, Eq. (lagdual) under Eq. (eqconst);
 *   - Keerthi's two-threshold SMO, Algorithm 1, with the gradient cache f of
 *     Eq. (fcache), its update Eq. (fup), the index sets Eq. (setinfo), the
 *     maximal-violating pair Eq. (bminmax), the stop test Eq. (kktterm) and
 *     the pair step Eqs. (alphaup)/(rho);
 *   - adaptive shrinking (Eq. (shrink), Algorithms 4 and 5, the counter
 *     heuristics of Section III-C and Table 3) with gradient reconstruction
 *     (Algorithm 6);
 *   - the classifier Eq. (classi) with the threshold b of Section III-A.
 *
 * Conventions shared by every call:
 *   - Kernel: K(x, z) = exp(-gamma * ||x - z||^2); gamma = 1 / (2 sigma^2)
 *     in the paper's notation (Section V-A).
 *   - f_i = sum_j alpha_j y_j K(x_i, x_j) - y_i (Eq. fcache).
 *   - Pair selection takes the lowest index on ties (both argmin and argmax).
 *   - Every call returns an int status (enum svm_status). No call aborts or
 *     throws; svm_last_error() gives a message for the last failing call of
 *     the calling thread.
 *   - All calls are synchronous with respect to the host unless stated: on
 *     return, outputs are written and the library's device work is done.
 *   - The library allocates its own device workspace (stream-ordered) and
 *     frees it before returning; inputs are only read, never kept.
 */
#ifndef SVM_GB300_H
#define SVM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------- status codes */
enum svm_status {
    SVM_OK = 0,
    SVM_NOT_CONVERGED = 1,   /* max_iter reached; outputs are valid but not optimal */
    SVM_PENDING = 2,         /* server: job still queued or running */
    SVM_ERR_ARG = -1,        /* invalid argument (see svm_last_error) */
    SVM_ERR_OOM = -2,        /* device or host allocation failed */
    SVM_ERR_BUDGET = -3,     /* server: job larger than the device-memory budget */
    SVM_ERR_TIMEOUT = -4,    /* a device-side wait exceeded its limit; the kernel
                                gave up and returned, the context stays usable */
    SVM_ERR_CUDA = -5,       /* a CUDA runtime call failed */
    SVM_ERR_CANCELLED = -6,  /* server: job cancelled */
    SVM_ERR_UNSUPPORTED = -7 /* valid input outside this build's limits
                                (e.g. more columns than the on-chip target rows hold) */
};

/* ------------------------------------------------------------- precision */
enum svm_precision {
    /* FP64 everywhere the result depends on it: inner products, kernel
     * values, f, the pair step, b and the gap. Inner products (and the
     * squared norms) of float rows are computed exactly in 128-bit integer
     * arithmetic and rounded once to the nearest double, when the nonzero
     * values of the matrix lie within 31 binades below the largest (rows
     * shorter than 2^17 entries; fewer binades for longer rows) and none is
     * subnormal; otherwise they are FP64 sums in row order. Binary (all
     * values 1.0) CSR input is detected at ingest and its kernel values are
     * taken from an exact FP64 table of exp(-gamma * k), k the integer
     * squared distance. */
    SVM_FP64 = 0,
    /* Inner products and exp in FP32 on BF16-rounded feature values (the
     * reconstruction and decision contractions on the tcgen05 tensor cores
     * with FP32 accumulation, for d <= 256); f, the pair step, b and the gap
     * stay FP64. */
    SVM_MIXED_BF16 = 1,
    /* The arithmetic of SVM_MIXED_BF16 with the contractions on the CUDA
     * cores instead of the tensor cores (a reference for the tensor-core
     * path, and the path used for d > 256). */
    SVM_MIXED_BF16_SIMT = 2
};

/* ----------------------------------------------------------- shrinking */
enum svm_shrink_kind {
    SVM_SHRINK_NONE = 0,     /* Table 3 row 1, "Original" (Algorithm 3's loop) */
    SVM_SHRINK_FIXED = 1,    /* counter h = value (Table 3 "random: k" rows, read
                                as the fixed constant k) */
    SVM_SHRINK_FRACTION = 2  /* counter h = ceil(value * N) (Table 3 "numsamples") */
};

enum svm_recon {
    SVM_RECON_SINGLE = 0,    /* Algorithm 5: one reconstruction, then no shrinking */
    SVM_RECON_MULTI = 1      /* shrinking throughout; reconstruct at first_factor*tau
                                the first time and at 2*tau afterwards */
};

/* CSR matrix. Row i holds columns indices[indptr[i] .. indptr[i+1]) with
 * values at the same positions. Column indices must be strictly increasing
 * within a row and in [0, d). values == NULL means every stored value is 1.0
 * (binary pattern). When on_device != 0 every pointer of the call that
 * receives this matrix (indptr, indices, values, labels, alpha, outputs of
 * length n or m) is device memory of the current device; otherwise host. */
typedef struct svm_csr {
    int64_t n;               /* rows */
    int64_t d;               /* columns */
    const int64_t *indptr;   /* n + 1 entries, indptr[0] == 0 */
    const int32_t *indices;  /* indptr[n] entries */
    const float *values;     /* indptr[n] entries, or NULL */
    int32_t on_device;
    int32_t reserved;
} svm_csr;

typedef struct svm_params {
    double C;                /* box bound, > 0 (Eq. eqconst) */
    double gamma;            /* RBF width, > 0 */
    double tau;              /* stop when b_low - b_up <= 2 tau (Eq. kktterm), > 0 */
    int64_t max_iter;        /* SMO step limit (<= 0: 100 * n + 1e6) */
    int32_t precision;       /* enum svm_precision */
    int32_t tie_break;       /* 0: lowest index (the only rule) */
    void *stream;            /* cudaStream_t to run on; NULL = legacy default stream */
    int32_t *trace;          /* optional HOST buffer: (i_up, i_low) of the first
                                trace_len steps, 2 ints per step; -1 if not reached */
    int64_t trace_len;
    int32_t flags;           /* bitwise OR of SVM_FLAG_* */
    int32_t ctas;            /* CTAs (= row segments) of the fused step; 0 = automatic:
                                one thread-block cluster of 16 CTAs when n <= 200,000
                                and its segments fit in shared memory, else one CTA
                                per SM (capped by n / 16); 16 asks for the single
                                cluster at any n; larger values are clamped */
    int32_t lanes_per_row;   /* lanes sharing one row in the row pass (rounded up to
                                a power of two <= 32); 0 = from the mean row length;
                                bit-mask rows always use one lane */
    int32_t cache_mb;        /* kernel-row cache in device memory (MiB) for inputs that
                                are not binary: 0 = automatic (FP64 precision only; up
                                to half the free memory, at most 32 GiB), < 0 = off,
                                > 0 = this budget (FP64 and mixed precision) */
    int32_t kernel;          /* enum svm_kernel_kind; 0 = RBF (Section V-A) */
    int32_t degree;          /* SVM_KERNEL_POLY: degree >= 1 */
    double coef0;            /* SVM_KERNEL_POLY / SVM_KERNEL_SIGMOID: offset */
    int64_t *active_trace;   /* optional HOST buffer: (step, active rows) after each of the
                                first active_trace_len shrink events (Eq. shrink), 2 int64
                                per event; -1 where no event happened */
    int64_t active_trace_len;
    const double *alpha0;    /* optional warm start (resume): n multipliers in X's memory
                                space, 0 <= alpha0 <= C and sum y alpha0 = 0 (within
                                1e-9 max(1, C n)); f is recomputed from them (Eq. fcache)
                                on the device; NULL = the usual start alpha = 0 */
} svm_params;

/* Kernels. RBF exp(-gamma ||x - z||^2) is the paper's (Section V-A); the
 * others are the standard ones Section V calls straightforward to use:
 * linear <x, z>, polynomial (gamma <x, z> + coef0)^degree, sigmoid
 * tanh(gamma <x, z> + coef0). They run on the FP64 and mixed row passes and
 * the CUDA-core contraction; binary inputs take the general (values) path,
 * and the tensor-core contraction, batches and the server are RBF only. */
typedef enum svm_kernel_kind {
    SVM_KERNEL_RBF = 0,
    SVM_KERNEL_LINEAR = 1,
    SVM_KERNEL_POLY = 2,
    SVM_KERNEL_SIGMOID = 3
} svm_kernel_kind;

typedef struct svm_kernel {
    int32_t kind;            /* enum svm_kernel_kind */
    int32_t degree;          /* polynomial degree >= 1 */
    double gamma;            /* > 0 */
    double coef0;
} svm_kernel;

/* Keep every row segment in global memory even when it would fit in the
 * SM's shared memory (the default holds rows, f, alpha and the index sets of
 * each segment on chip for the whole solve when they fit). */
#define SVM_FLAG_STREAM_ROWS 1
/* Record the SM cycles one CTA spends in each phase of a step
 * (svm_stats.phase_ms, converted at the device's maximum clock). */
#define SVM_FLAG_PHASE_TIMES 2
/* Exchange the per-step candidates of all CTAs through global memory only
 * (by default the CTAs form one cluster of 16 that reduces through
 * distributed shared memory alone, or clusters of 8 whose leaders exchange
 * through global memory). */
#define SVM_FLAG_NO_CLUSTERS 4
/* Binary input (every stored value 1.0) with d <= 256 is read in the row
 * pass as one bit mask per row (16 or 32 bytes), the squared distance to
 * x_up / x_low being the popcount of an XOR; this flag keeps the CSR column
 * gather instead. The results are identical either way. */
#define SVM_FLAG_CSR_ROWS 8
/* Second-order working-set selection (the paper's future work, Section VI;
 * Fan, Chen and Lin, JMLR 6, 2005): i_up as in Eq. (bminmax), i_low the row
 * t of I_low with f_t > f_up of largest gain (f_t - f_up)^2 / eta_ut,
 * eta_ut = K_uu + K_tt - 2 K_ut (1e-12 when not positive), over the active
 * rows, lowest index on ties. The stopping test (Eq. kktterm), the shrink
 * rule (Eq. shrink) and the reported b_up / b_low keep the first-order
 * extremes. Each step adds a sweep over the active rows and a second
 * candidate exchange. svm_train and svm_train_fixed_workspace only. */
#define SVM_FLAG_WSS2 16
/* With shrinking, a launch over a problem that is not already one on-chip
 * cluster ends once fewer than three quarters of its rows are active; the active rows
 * are gathered (in index order) into a smaller problem whose launch shape is
 * chosen again, and the state is scattered back when it ends. The steps are
 * the same either way (same pairs, same arithmetic); this flag turns the
 * re-layout off. */
#define SVM_FLAG_NO_RELAYOUT 32
/* Kernel rows on the tensor cores (SVM_MIXED_BF16, RBF, d <= 256, no
 * kernel-row cache): tiles of 16 active rows against the two target rows
 * (BF16 inputs, FP32 accumulation) from a dense BF16 copy of the rows. Used
 * automatically when the rows are dense enough (mean stored entries per row
 * >= 32 and >= half of d rounded up to 32, d <= 128); SVM_FLAG_TENSOR_ROWS
 * asks for it wherever it applies, SVM_FLAG_CUDA_CORE_ROWS keeps the CSR row
 * pass on the CUDA cores (same arithmetic type, another summation order). */
#define SVM_FLAG_CUDA_CORE_ROWS 64
#define SVM_FLAG_TENSOR_ROWS 128
/* Gradient reconstruction (Algorithm 6) always as the full sum over the
 * support vectors. By default, when the launch over all rows that follows a
 * multiple-reconstruction restart ends at its first shrink event and its
 * active rows are gathered by the re-layout, the rows shrunk there (whose f
 * was exact at that moment) are reconstructed as that f plus the sum over the
 * gathered rows whose alpha changed since: the same value up to rounding
 * order, over far fewer terms. CUDA-core contraction only (FP64, binary and
 * SVM_MIXED_BF16_SIMT inputs); svm_stats.incremental_recons counts them. */
#define SVM_FLAG_FULL_RECON 256

typedef struct svm_shrink_policy {
    int32_t kind;            /* enum svm_shrink_kind */
    int32_t recon;           /* enum svm_recon */
    double value;            /* k (FIXED) or fraction of N (FRACTION) */
    double first_factor;     /* first reconstruction when the active gap <=
                                first_factor * tau; <= 0 means 20 (Algorithm 5) */
} svm_shrink_policy;

/* The paper's three classes of shrinking heuristics (Section IV, Table 3),
 * with multiple reconstructions: aggressive (counter 5% of N), average (10%)
 * and lazy (50%). Usable as initialisers:
 *   svm_shrink_policy p = SVM_SHRINK_AGGRESSIVE; */
#define SVM_SHRINK_AGGRESSIVE {SVM_SHRINK_FRACTION, SVM_RECON_MULTI, 0.05, 20.0}
#define SVM_SHRINK_AVERAGE {SVM_SHRINK_FRACTION, SVM_RECON_MULTI, 0.10, 20.0}
#define SVM_SHRINK_LAZY {SVM_SHRINK_FRACTION, SVM_RECON_MULTI, 0.50, 20.0}

typedef struct svm_stats {
    int64_t iters;           /* SMO steps */
    int64_t shrink_events;
    int64_t reconstructions;
    int64_t final_active;    /* active-set size when the last phase ended */
    int64_t n_sv;            /* alpha > 0 */
    int64_t n_bound;         /* alpha == C */
    int64_t row_visits;      /* sum over steps of the active-set size */
    double b_up, b_low;      /* Eq. (bminmax) over all samples at exit */
    double objective;        /* dual objective W at exit */
    double ms_total;         /* wall time of the call */
    double ms_smo;           /* device time in the fused SMO kernel(s) */
    double ms_recon;         /* device time in reconstruction (Algorithm 6) */
    int32_t binary_input;    /* 1 when the binary-pattern path was used */
    int32_t launches;        /* kernel launches issued by the call */
    int32_t resident;        /* 1 when row segments were held in shared memory */
    int32_t ctas;            /* CTAs (= row segments) of the fused step */
    int32_t lanes_per_row;   /* lanes that share one row in the row pass */
    int32_t cluster_size;    /* CTAs per thread-block cluster of the fused step */
    double phase_ms[8];      /* with SVM_FLAG_PHASE_TIMES: time of CTA 0 per step
                                phase, summed over steps: target rows, pair step
                                (FP64 part), row pass + CTA reduction, publish,
                                grid exchange, other, pair step (K(up,low) part),
                                second-order gain sweep and exchange */
    double cta_busy_ms_min;  /* with SVM_FLAG_PHASE_TIMES: least and most time a */
    double cta_busy_ms_max;  /* CTA spent from step start to publishing its candidate */
    int32_t bit_rows;        /* 1 when the row pass read binary rows as bit masks */
    int32_t cache_slots;     /* kernel rows the cache holds (0: no cache) */
    int64_t cache_hits;      /* steps x sides whose kernel row came from the cache */
    int64_t cache_misses;    /* ... that were computed (and stored) */
    int64_t relayouts;       /* active-set re-layouts (see SVM_FLAG_NO_RELAYOUT) */
    int32_t row_tiles;       /* 1 when the kernel rows ran on the tensor cores */
    int32_t incremental_recons;   /* reconstructions done incrementally (SVM_FLAG_FULL_RECON) */
} svm_stats;

/*
 * svm_train -- solve the dual QP (Eq. lagdual) by SMO (Algorithm 1) with the
 * given shrinking policy (Algorithms 4-6).
 *   X         training rows (n >= 2, d >= 1); see svm_csr for memory space
 *   y         n labels, +1 or -1, both classes present (same space as X)
 *   params    C, gamma, tau, max_iter, precision, stream, trace
 *   policy    shrinking policy; NULL = SVM_SHRINK_NONE
 *   alpha_out n doubles written with the multipliers (same space as X;
 *             caller-owned)
 *   b_out     threshold b of Section III-A (host)
 *   iters_out SMO steps (host, may be NULL)
 *   stats     optional (host, may be NULL)
 * Returns SVM_OK, SVM_NOT_CONVERGED (outputs valid), or an error; on error the
 * outputs are unspecified.
 */
int svm_train(const svm_csr *X, const int8_t *y, const svm_params *params,
              const svm_shrink_policy *policy, double *alpha_out, double *b_out,
              int64_t *iters_out, svm_stats *stats);

/*
 * svm_decision -- Eq. (classi) before the sign:
 *   out[k] = sum_{j : alpha_j > 0} alpha_j y_j K(x_j, z_k) - b.
 *   X, y, alpha  training rows, labels and multipliers (space of X)
 *   Z            m query rows with Z->d == X->d (space of Z; out in that space)
 *   precision    enum svm_precision (SVM_MIXED_BF16 uses the tensor cores)
 *   stream       cudaStream_t or NULL
 */
int svm_decision(const svm_csr *X, const int8_t *y, const double *alpha, double b,
                 double gamma, const svm_csr *Z, int32_t precision, void *stream,
                 double *out);

/*
 * svm_decision_kernel -- svm_decision for any svm_kernel (the RBF kernel
 * gives the same values as svm_decision). Non-RBF kernels use the CUDA-core
 * contraction in FP64 or mixed precision.
 */
int svm_decision_kernel(const svm_csr *X, const int8_t *y, const double *alpha, double b,
                        const svm_kernel *kernel, const svm_csr *Z, int32_t precision,
                        void *stream, double *out);

/* ------------------------------------------------------ resident model */

/* A trained model held on the device: the support vectors (the rows of X
 * with alpha > 0, Section III-A's zeta), their coefficients alpha_i y_i, the
 * threshold b and the kernel, so that the classifier of Eq. (classi) can be
 * evaluated on new queries without re-reading the training rows or alpha.
 * The handle owns its device memory, on the device current at creation. */
typedef struct svm_model svm_model;

/*
 * svm_model_create -- gather the support vectors of a trained problem.
 *   X, y, alpha   the training rows, labels and multipliers of svm_train
 *                 (one memory space, as in svm_decision; read, not kept)
 *   b, kernel     threshold and kernel of the training
 *   precision     arithmetic of later decisions (enum svm_precision)
 *   out           receives the handle (NULL on error)
 * Errors: SVM_ERR_ARG (NULL pointers, bad kernel, inputs as for svm_decision),
 * SVM_ERR_OOM, SVM_ERR_CUDA. Synchronous.
 */
int svm_model_create(const svm_csr *X, const int8_t *y, const double *alpha, double b,
                     const svm_kernel *kernel, int32_t precision, void *stream, svm_model **out);

/*
 * svm_model_decision -- Eq. (classi) before the sign for the m rows of Z:
 * out[q] = sum over support vectors k of alpha_k y_k K(x_k, z_q) - b; the
 * same values as svm_decision_kernel on the model's training inputs.
 * Z->d must equal the model's d; the current device must be the model's.
 * out (m doubles) is in Z's memory space. Synchronous; calls on one model
 * may overlap (the model is only read).
 */
int svm_model_decision(const svm_model *model, const svm_csr *Z, void *stream, double *out);

/* Support vectors, columns and threshold of a model (each output nullable). */
int svm_model_info(const svm_model *model, int64_t *n_sv, int64_t *d, double *b);

/* Releases the model and its device memory (NULL is accepted). */
int svm_model_free(svm_model *model);

/* ------------------------------------------------------------ batching */

/* One training job of a batch: a two-class subproblem over rows of the shared
 * matrix (e.g. one class pair of a one-vs-one split, with its own C and
 * gamma). Pointers are in the memory space of the batch's matrix. */
typedef struct svm_job {
    int64_t n_rows;          /* rows in the subproblem (>= 2) */
    const int32_t *rows;     /* n_rows row ids of the matrix; NULL = rows 0 .. n_rows-1 */
    const int8_t *y;         /* n_rows labels, +1 / -1, both present */
    double C, gamma, tau;    /* as in svm_params */
    int64_t max_iter;        /* <= 0: 100 * n_rows + 1e6 */
    double *alpha_out;       /* n_rows multipliers (caller-owned) */
} svm_job;

typedef struct svm_result {
    double b;                /* threshold of Section III-A */
    double b_up, b_low;      /* Eq. (bminmax) at exit */
    double objective;        /* dual objective W */
    int64_t iters;
    int32_t status;          /* SVM_OK or SVM_NOT_CONVERGED */
    int32_t n_sv;
} svm_result;

typedef struct svm_batch_config {
    int32_t precision;       /* enum svm_precision (tensor cores are not used here) */
    int32_t cluster_size;    /* in/out: CTAs that share one job (1..16, power of
                                two); 0 = picked by svm_batch_autotune */
    int32_t lanes_per_row;   /* in/out: lanes per row in the row pass; 0 = autotuned */
    int32_t clusters;        /* jobs in flight at once; 0 = as many as fit */
    void *stream;            /* cudaStream_t or NULL */
    double ms_kernel;        /* out: device time of the batched launch */
    double ms_total;         /* out: wall time of the call */
    int64_t iters_total;     /* out: SMO steps summed over the jobs */
    int32_t clusters_used;   /* out */
    int32_t reserved;
} svm_batch_config;

/*
 * svm_train_batch -- train every job (plain SMO, Algorithm 1, per job) in one
 * persistent launch: thread-block clusters take jobs from a device work-list;
 * each job's rows are split over the CTAs of one cluster, which exchange
 * their candidates through distributed shared memory. X is ingested once for
 * all jobs. Results and multipliers are those each job would get alone with
 * svm_train at the same precision (no shrinking). Returns SVM_OK,
 * SVM_NOT_CONVERGED (some job hit max_iter) or an error.
 */
int svm_train_batch(const svm_csr *X, const svm_job *jobs, int32_t n_jobs,
                    svm_batch_config *config, svm_result *results);

/*
 * svm_batch_autotune -- choose cluster_size and lanes_per_row for this matrix
 * and these jobs by timing each candidate shape on a sample of at most 64
 * jobs capped at 300 steps, and write the fastest into *config. Fields the
 * caller set to non-zero values are kept.
 */
int svm_batch_autotune(const svm_csr *X, const svm_job *jobs, int32_t n_jobs,
                       svm_batch_config *config);

/* ------------------------------------------------------------- serving */

/* A training server: jobs of any n and d arrive over time, are admitted while
 * a slot and the device-memory budget allow, and run concurrently on the
 * device (continuous batching): a persistent engine kernel made of
 * thread-block clusters takes admitted jobs from a ring the host extends
 * while the engine runs; each job's matrix, alpha and f stay resident on the
 * device until it finishes. Every job is the plain solve of Algorithm 1; its
 * result is the one svm_train gives alone at the same precision. */
typedef struct svm_server svm_server;

typedef struct svm_server_config {
    size_t budget_bytes;     /* device memory the server may hold for jobs */
    int32_t max_slots;       /* jobs on the device at once (<= 1024; 0 = 64) */
    int32_t precision;       /* SVM_FP64 or SVM_MIXED_BF16 */
    int32_t cluster_size;    /* CTAs per job (power of two <= 16; 0 = 16) */
    int32_t lanes_per_row;   /* 0 = 2 */
    int32_t max_d;           /* widest job accepted (0 = 2048) */
    int32_t reserved;
} svm_server_config;

typedef struct svm_server_times {
    double submit_to_admit_ms;
    double admit_to_done_ms;
    double submit_to_done_ms;   /* time to model */
} svm_server_times;

typedef struct svm_server_info {
    size_t bytes_in_use, budget_bytes;
    int32_t queued, running;
    int32_t clusters, cluster_size;   /* engine: jobs that can run at once, CTAs each */
    int64_t engine_launches;
} svm_server_info;

/* Create a server on the current device (starts its host worker thread). */
int svm_server_create(const svm_server_config *config, svm_server **out);
/* Queue a job. X and y are host buffers and are copied before the call
 * returns. SVM_ERR_BUDGET if the job alone exceeds the budget. */
int svm_server_submit(svm_server *srv, const svm_csr *X, const int8_t *y,
                      const svm_params *params, uint64_t *ticket);
/* Non-blocking: SVM_PENDING while queued or running; otherwise the job's
 * status, and res / alpha_out (n doubles) / times are filled (each may be
 * NULL) and the ticket is released. */
int svm_server_poll(svm_server *srv, uint64_t ticket, svm_result *res, double *alpha_out,
                    svm_server_times *times);
/* As svm_server_poll, waiting up to timeout_s seconds for the job. */
int svm_server_wait(svm_server *srv, uint64_t ticket, double timeout_s, svm_result *res,
                    double *alpha_out, svm_server_times *times);
/* Cancel: a queued job ends with SVM_ERR_CANCELLED; a running job finishes
 * on the device and then reports SVM_ERR_CANCELLED. */
int svm_server_cancel(svm_server *srv, uint64_t ticket);
int svm_server_stats(svm_server *srv, svm_server_info *info);
/* Stop the server: running jobs finish, queued jobs are dropped. */
int svm_server_destroy(svm_server *srv);

/*
 * svm_train_fixed_workspace -- the plain solve of svm_train (no shrinking,
 * SVM_FP64) without any device allocation. The paper has no counterpart to
 * this call; it exists for callers that cannot allocate device memory while
 * they train: code that runs inside a memory pool capped or owned by someone
 * else, a latency-bound loop that must not wait on the allocator, or a
 * process that reserved the whole device before it started.
 *
 * All scratch (gradient, index sets, active lists, exchange slots, tables,
 * reductions) lives in one 4 MiB file-scope device array. CUDA places it in
 * a GPU's memory when the library's code is first loaded on that GPU: under
 * lazy module loading (CUDA's default) that is the first call of this
 * library that runs device work there, not the moment the shared object is
 * opened. It then stays until the process exits. A caller that caps or
 * reserves device memory should therefore make one call first (a small
 * warm-up problem through this entry point) on each GPU it will use. The
 * caller passes the inputs and the output buffer in device memory:
 *   X         device CSR (X->on_device must be 1), 2 <= n <= 131072 rows,
 *             d < 2^31, at most 4096 entries in a row
 *   y         n device labels (+1 / -1)
 *   params    C, gamma, tau, max_iter, stream; precision must be SVM_FP64;
 *             flags other than SVM_FLAG_WSS2 are ignored, as are trace,
 *             ctas and lanes_per_row
 *   alpha_out n doubles of device memory, written with the multipliers
 *   b_out     host double; iters_out host int64 (may be NULL)
 * Larger problems return SVM_ERR_UNSUPPORTED with a message naming the
 * limit; d >= 2^31 returns SVM_ERR_ARG before any device work. Binary input
 * (every stored value 1.0) whose distance tables do not fit in shared
 * memory takes the FP64 row pass, as in svm_train; it then needs explicit
 * values (values == NULL there gives SVM_ERR_UNSUPPORTED). Other results are
 * those of svm_train.
 *
 * The first call on each device looks up the device address of the array
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Every call uses the same array and starts by re-initialising the parts it
 * reads, so consecutive calls are independent; calls whose device work
 * overlaps (two host threads, or two streams) race on the array and must
 * not be issued.
 */
int svm_train_fixed_workspace(const svm_csr *X, const int8_t *y, const svm_params *params,
                              double *alpha_out, double *b_out, int64_t *iters_out);

/* Number of CUDA kernels this library has launched in this process (all
 * threads, all calls), for accounting of device work. */
int64_t svm_kernel_launches(void);

/* Failure-handling check (the paper has no counterpart: its outer-loop flag
 * is never set, and this library bounds every device-side wait instead).
 * Runs, on the device, the bounded wait that the fused step uses for its
 * candidate exchange, on an mbarrier that nothing completes, with the given
 * limit:
 *   limit_ns  1e6 .. 5e9 (1 ms .. 5 s)
 *   stream    cudaStream_t (NULL = legacy default stream)
 * Returns SVM_ERR_TIMEOUT when the wait gave up (the expected outcome; the
 * CUDA context stays usable), SVM_OK if it did not, SVM_ERR_ARG for a limit
 * out of range. Synchronous. */
int svm_diag_wait_timeout(int64_t limit_ns, void *stream);

/* Measurement aid (the paper has no counterpart): the rate of the SFU's
 * exp2 instruction over the whole device, from a kernel of independent
 * ex2.approx chains (the instruction of the RBF contraction's epilogue), so
 * that the contraction can be reported against the exp rate it is bound by.
 * ex2_per_s receives instructions per second. Synchronous. */
int svm_diag_sfu_rate(double *ex2_per_s, void *stream);

/* Message for the last failing call on this thread ("" if none). */
const char *svm_last_error(void);

/* Library version string. */
const char *svm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SVM_GB300_H */
