/*
 * rtdetmcd.h - C ABI of the GB300 (sm_103a) RT-DetMCD engine.
 *
 * RT-DetMCD is the real-time deterministic Minimum Covariance Determinant
 * outlier detector of De Ketelaere, Hubert, Raymaekers, Rousseeuw and Vranckx
 * (arXiv 1910.05615).  Given n observations x_i in R^p (the n x p data matrix
 * X of Section 2) and a coverage h with [(n+p+1)/2] <= h < n (Section 2.1),
 * it returns a robust centre and scatter and flags as outliers the rows whose
 * robust distance exceeds the cutoff sqrt(chi2_{p,q}), q = 0.975 by default
 * (Section 2.1).
 *
 * Conventions shared by every entry point
 *   - Row data are float32, row-major, row stride `ld` floats (ld >= p).
 *     Every data / output pointer may be device memory or host memory
 *     (pageable or pinned); host buffers are staged through the workspace.
 *     Device memory must belong to the current device (RTD_EINVAL for
 *     another device's memory).
 *   - `workspace` is device memory owned by the caller, at least the size
 *     returned by the matching *_workspace_size call, 256-byte aligned.  No
 *     entry point allocates device memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is issued on that stream; the calls return after the
 *     stream has finished their work, so outputs are valid on return.
 *   - The return value is a status code (RTD_OK = 0).  Invalid arguments are
 *     rejected before any device work.  Data-dependent failures (non-finite
 *     input, degenerate columns, every start ill-conditioned) are detected on
 *     the device and returned; warnings are reported in rtd_result.warnings.
 *   - p <= RTD_MAX_P, n < 2^31.
 */
#ifndef RTDETMCD_H
#define RTDETMCD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RTD_MAX_P 64
#define RTD_MAX_BLOCKS 1024   /* largest number of blocks q of Section 4 */

/* status codes */
#define RTD_OK            0
#define RTD_EINVAL        1  /* bad argument: h out of range, p < 1 or > 64, ld < p, n <= 2p, ... */
#define RTD_ENONFINITE    2  /* a NaN or Inf in the rows */
#define RTD_EILLCOND      3  /* every start of every block was dropped (Section 3.3 step 2 / Section 3.4) */
#define RTD_EDEGENERATE   4  /* zero univariate MCD scale, or a fitted scatter not positive definite */
#define RTD_EWORKSPACE    5  /* workspace too small or misaligned */
#define RTD_ECUDA         6  /* a CUDA runtime error */
#define RTD_EINTERNAL     7  /* an internal consistency check failed */

/* warning bits (rtd_result.warnings) */
#define RTD_WARN_MAXITER        1  /* a C-step chain stopped at max_csteps */
#define RTD_WARN_DROPPED_START  2  /* at least one start was dropped as ill-conditioned */
#define RTD_WARN_CSTEP_REFUSED  4  /* the condition monitor stopped a chain (Section 3.4) */
#define RTD_WARN_NO_BLOCK_FIT   8  /* at least one block had no fit */

/* arithmetic of the row passes (distances, Grams, sort keys) */
#define RTD_FP64 0   /* plain FP64 form */
#define RTD_FP32 1   /* FP32 row passes, FP64 p x p algebra, FP64 recompute near every threshold */
#define RTD_BF16 2   /* the FP32 form with the Grams of the starts and C-steps on the tensor
                        cores: rows centred in FP32 and split into BF16 high, middle and low
                        parts (24 significant bits), the six leading partial products with FP32
                        accumulation, compensated FP32 sums every 128 rows; the reweighting Gram
                        stays on the FP32 CUDA-core path; 25 <= p <= 48 (RTD_EINVAL otherwise) */

typedef struct {
    int32_t  precision;            /* RTD_FP32 (default), RTD_FP64 or RTD_BF16 */
    int32_t  omega;                /* eq. partitionsize, default 4096 */
    int32_t  q_override;           /* number of blocks, at most RTD_MAX_BLOCKS (RTD_EINVAL above);
                                      0 = q = min(max(floor(n/(p omega)), 1), RTD_MAX_BLOCKS) */
    int32_t  max_csteps;           /* C-step cap per start, default 100 */
    double   cutoff_q;             /* chi-square quantile of the cutoff, default 0.975 */
    double   kappa_max;            /* condition threshold, default 1000 (Sections 3.3, 3.4) */
    uint64_t seed;                 /* random partition of Section 4, default 0 */
    int32_t  reweight_consistency; /* 0: plain covariance of the reweighted set;
                                      1 (default): times 0.975 / F_{chi2_{p+2}}(chi2_{p,0.975});
                                      2: times c(|W|/n) at the kept fraction */
    int32_t  select_path;          /* FP32 form, C-step selection from the second step on:
                                      0 (default) rows classified against a threshold window
                                      predicted from the last steps, histogram path when it misses;
                                      1 histogram path at every step;
                                      2 window of the smallest half-width (misses exercise the
                                      histogram path).  All three select the same h-subset. */
    /* optional per-row output (nullable, device or host, n bytes, original row
       order): bit0 = row is in the final h-subset of its block's chosen start,
       bit1 = row is in the reweighting set W. */
    uint8_t* subset_out;
    /* optional diagnostics (nullable, device or host), rtdetmcd_diag_size()
       bytes of doubles laid out as documented at rtdetmcd_diag_size. */
    double*  diag_out;
    /* optional stage profile (nullable, host), filled on return */
    struct rtd_profile* profile;
    /* optional warm start (both or neither; host, X units): the final mu (p)
       and Sigma (p x p, row-major) of an earlier fit, used as the input to
       step 3 of Section 4 (end of Section 4).  Every block then runs one
       C-step chain from it; the univariate standardisation, the initial
       estimators and their refinement (Sections 3.1-3.3) are skipped, and Z
       is standardised by the warm fit's centre and diagonal.  Rejected with
       RTD_EINVAL unless finite with a positive diagonal. */
    const double* init_mu;
    const double* init_sigma;
    int32_t  dist_path;            /* FP32 form, C-step distances from the second step on:
                                      0 (default) CUDA-core FP32 FMAs;
                                      1 tcgen05 tensor cores with split-TF32 operands (p <= 40;
                                      wider rows take the CUDA-core pass).  Both take the same
                                      decisions (every threshold decision near the FP32 error is
                                      made in FP64). */
    int32_t  graph;                /* 0 (default): stream launches, the host reads a status word
                                      between the stages and after every C-step;
                                      1: the whole fit as one captured CUDA graph with its control
                                      flow on the device (conditional nodes: the C-step loop runs
                                      while a chain iterates, later stages only if no error), kept
                                      per host thread and relaunched when the same arguments come
                                      again.  Needs device rows and outputs, no profile and no warm
                                      start (the stream path is taken otherwise). */
    int32_t  autotune;             /* rtdetmcd_fit_batch with graph = 1: 1 (default) tunes each class
                                      of frames without a tuned launch shape first (see
                                      rtdetmcd_autotune); 0 uses the tuned or default shapes */
    int32_t  reserved1;
} rtd_options;

/* Stages of a fit, for rtd_profile. */
#define RTD_STAGE_PARTITION   0   /* random partition copy (Section 4) */
#define RTD_STAGE_UNIVARIATE  1   /* column univariate MCD (Sections 3.1, 4) */
#define RTD_STAGE_STARTS      2   /* wrapping and GSSCM scatters (Section 3.2) */
#define RTD_STAGE_REFINE      3   /* refinement (Section 3.3) */
#define RTD_STAGE_CPREP       4   /* Cholesky and condition monitor per C-step (Section 3.4) */
#define RTD_STAGE_CDIST       5   /* C-step distances + top-digit histogram */
#define RTD_STAGE_CSELECT     6   /* radix select of the h_b smallest */
#define RTD_STAGE_CUPDATE     7   /* membership update and Gram update (Section 3.5) */
#define RTD_STAGE_AGGREGATE   8   /* block choice, median, KL, pooling (Section 4 steps 4-7) */
#define RTD_STAGE_REWEIGHT    9   /* reweighting (steps 8-9) */
#define RTD_STAGE_FINAL      10   /* final distances and flags (step 10) */
#define RTD_STAGE_SORT       11   /* segmented radix sorts (timed apart from the stages above) */
#define RTD_NSTAGES          12

/* Per-stage device time (CUDA events recorded on the fit's stream around
   each stage), algorithmic bytes (each row and key read or written once per
   pass) and kernel launches of one rtdetmcd_fit call. */
typedef struct rtd_profile {
    double  ms[RTD_NSTAGES];
    double  bytes[RTD_NSTAGES];
    int64_t launches[RTD_NSTAGES];
    int32_t csteps;        /* C-step iterations run (all chains in lockstep) */
    int32_t win_steps;     /* chain steps whose selection used the predicted window (FP32 form) */
    int32_t win_miss;      /* of those, steps whose window missed (histogram path taken) */
    int32_t reserved;
    int64_t sel_cand;      /* selection candidates listed, summed over chain steps */
    int64_t sel_band;      /* rows decided in FP64 inside the band, summed over chain steps */
    /* algorithmic floating-point operations per stage (an FMA counts 2);
       filled for the C-step distances: p (p + 3) per row and active chain
       (the triangular product and the squares), in the form's precision */
    double  flops[RTD_NSTAGES];
} rtd_profile;

typedef struct {
    int32_t status;        /* same as the return value */
    int32_t warnings;      /* RTD_WARN_* bits */
    int32_t p, q;          /* dimension, number of blocks */
    int64_t n, m, h, h_b;  /* rows, rows per block, coverage, coverage per block */
    double  mu[RTD_MAX_P];                 /* reweighted centre, X units */
    double  sigma[RTD_MAX_P * RTD_MAX_P];  /* reweighted scatter, row-major p x p (stride p) */
    double  mu_raw[RTD_MAX_P];             /* raw (aggregated) centre */
    double  sigma_raw[RTD_MAX_P * RTD_MAX_P];
    double  logdet;        /* log det sigma */
    double  logdet_raw;
    double  cutoff_d2;     /* chi2_{p,cutoff_q} */
    int64_t n_flagged;     /* rows with d2 > cutoff_d2 */
    int64_t n_reweight;    /* |W| */
    int32_t csteps_max;    /* largest number of C-steps over all chains */
    int32_t chains_ok;     /* chains that produced a fit */
    double  c_rew;         /* factor of the reweighted scatter: sigma = c_rew * (sample covariance of W) */
} rtd_result;

/* Fill *opt with the defaults listed above. */
void rtdetmcd_default_options(rtd_options* opt);

/* Bytes of workspace rtdetmcd_fit needs for an n x p problem under *opt
   (opt may be NULL for the defaults).  Returns 0 for invalid n, p. */
size_t rtdetmcd_workspace_size(int64_t n, int32_t p, const rtd_options* opt);

/* Bytes of diagnostics written to opt->diag_out for q blocks (q as in
   rtd_result.q).  Layout, all doubles, Z = standardised units (Section 4,
   eq. standardization):
     [0, p)          mu_uni   (univariate MCD location of each column)
     [p, 2p)         sigma_uni
     then for each chain c = 2 l + k (block l, start k = 0 wrapping,
     k = 1 GSSCM), a record of 3 p^2 + 2 p + 6 doubles:
        S_init[p^2]      initial scatter S~_k (Section 3.2)
        Sigma_start[p^2] refined start Sigma_k (Section 3.3)
        mu_start[p]
        Sigma[p^2]       final C-step scatter Lambda/(h_b-1), without c(alpha)
        mu[p]
        logdet, steps, status (0 ok, 1 dropped at refinement, 2 refused by the
        condition monitor before any step, 3 max steps), full_recomputes,
        last_swaps, kappa1
     then for each block l: chosen start (-1 none), KL deviation, kept (0/1). */
size_t rtdetmcd_diag_size(int32_t p, int32_t q);

/*
 * Full RT-DetMCD fit (Section 4, steps 1-10, with the Section 3 serial
 * improvements inside each block; q = 1 is the serial algorithm).
 *   X          n rows of p floats, stride ld
 *   h          coverage, [(n+p+1)/2] <= h < n
 *   opt        options (NULL = defaults)
 *   out        host pointer, filled on return (required)
 *   d2_out     nullable, n floats: final squared robust distances, original order
 *   flags_out  nullable, n bytes: 1 where d2 > cutoff_d2 (Section 4 step 10)
 */
int rtdetmcd_fit(const float* X, int64_t n, int32_t p, int64_t ld, int64_t h,
                 const rtd_options* opt, void* workspace, size_t ws_bytes,
                 void* stream, rtd_result* out, float* d2_out, uint8_t* flags_out);

/*
 * The fit in stages, for one fit sharded over G processes (one GPU each).
 * Section 4 groups into stages whose exchanges are small:
 *   - the univariate MCD of each column (Section 3.1, eq. standardization):
 *     columns are independent;
 *   - steps 2-4 (starts, refinement, C-steps, choice of start) of each block:
 *     blocks are independent (the paper runs one thread per block);
 *   - steps 5-7 read only the q block fits (p + p^2 + 2 doubles each);
 *   - steps 8-9 sum over the rows of all blocks: count, sum and centred
 *     cross-products of the reweighting set (1 + p + p^2 doubles);
 *   - step 10 treats each row alone.
 * A process takes a range of columns, a range of blocks and a range of rows;
 * between the stages the processes all-gather the column results and the
 * block fits and sum the moments.  Called with the whole ranges in one process
 * the stages give rtdetmcd_fit's results, up to the order of the FP64 sums of
 * the moments (which can move the reweighted fit by a few units in the last
 * place).
 * Every stage call: X is the whole n x p matrix (device or host; host rows are
 * copied in every call), h and opt as for rtdetmcd_fit and equal in every call
 * and process (opt->init_mu must be NULL; graph, subset_out, diag_out and
 * profile are ignored); the workspace has at least
 * rtdetmcd_workspace_size(n, p, opt) bytes; results may go to host or device
 * memory; the call returns when they are written.  Returns RTD_EINVAL for a
 * range outside [0, p), [0, q) or [0, n) or a missing pointer, and the status
 * of the stage's data otherwise (RTD_ENONFINITE, RTD_EDEGENERATE, ...).
 */
#define RTD_BLOCK_FIT_DOUBLES(p) (2 + (p) + (p) * (p))
#define RTD_MOMENT_DOUBLES(p) (1 + (p) + (p) * (p))

/* Block count q and rows per block m of the partition of Section 4
   (eq. partitionsize) for these arguments. */
int rtdetmcd_partition(int64_t n, int32_t p, int64_t h, const rtd_options* opt, int32_t* q, int64_t* m);

/* Univariate reweighted MCD (Section 3.1) of columns [col_lo, col_hi) over
   all n rows, and the non-finite check of those columns: uni_out receives
   2 (col_hi - col_lo) doubles, the locations then the scales (mu_uni, s_uni
   of eq. standardization). */
int rtdetmcd_standardize(const float* X, int64_t n, int32_t p, int64_t ld, int64_t h, const rtd_options* opt,
                         int32_t col_lo, int32_t col_hi, void* workspace, size_t ws_bytes, void* stream,
                         double* uni_out);

/* Section 4 steps 2-4 for blocks [blk_lo, blk_hi) of the partition, with the
   standardisation uni (2p doubles: all locations, then all scales).
   fits_out receives one record of RTD_BLOCK_FIT_DOUBLES(p) doubles per block:
     chosen start (0 wrapping, 1 GSSCM; -1 when neither gave a fit),
     log det Sigma_l, mu_l[p], Sigma_l[p^2] row-major
   in Z units, Sigma_l = Lambda/(h_b - 1) without c(alpha).  An empty range
   does nothing. */
int rtdetmcd_fit_blocks(const float* X, int64_t n, int32_t p, int64_t ld, int64_t h, const rtd_options* opt,
                        const double* uni, int32_t blk_lo, int32_t blk_hi, void* workspace, size_t ws_bytes,
                        void* stream, double* fits_out);

/* Steps 5-7 from the records of all q blocks (fits, block order), then the
   step-8 distances to the raw fit of the rows of blocks [blk_lo, blk_hi):
   moments_out receives RTD_MOMENT_DOUBLES(p) doubles, the count of the rows
   of the reweighting set W, the sum of x - c and the sum of (x - c)(x - c)^T
   over them (row-major), with c the raw centre in X units (the same in every
   process, since steps 5-7 are).  An empty range gives zeros.
   RTD_EILLCOND if no block has a fit; RTD_EINVAL for a malformed record. */
int rtdetmcd_reweight_moments(const float* X, int64_t n, int32_t p, int64_t ld, int64_t h, const rtd_options* opt,
                              const double* uni, const double* fits, int32_t blk_lo, int32_t blk_hi,
                              void* workspace, size_t ws_bytes, void* stream, double* moments_out);

/* Step 9 from the moments summed over all blocks (every process's
   rtdetmcd_reweight_moments added entrywise), then step 10 for the original
   rows [row_lo, row_hi): out (host) as for rtdetmcd_fit, with n_flagged
   counting those rows only and csteps_max, chains_ok zero; d2_out and
   flags_out (nullable) receive row_hi - row_lo entries. */
int rtdetmcd_reweight_finish(const float* X, int64_t n, int32_t p, int64_t ld, int64_t h, const rtd_options* opt,
                             const double* uni, const double* fits, const double* moments, int64_t row_lo,
                             int64_t row_hi, void* workspace, size_t ws_bytes, void* stream, rtd_result* out,
                             float* d2_out, uint8_t* flags_out);

/* Largest number of concurrent streams of rtdetmcd_fit_batch. */
#define RTD_BATCH_MAX_STREAMS 64

/* Bytes of workspace rtdetmcd_fit_batch needs: one slice per stream, each
   sized for the largest frame (h taken at its lower bound does not change the
   size). */
size_t rtdetmcd_fit_batch_workspace_size(int32_t nframes, const int64_t* n, const int32_t* p,
                                         const rtd_options* opt, int32_t nstreams);

/*
 * Many independent fits (Section 4 steps 1-10 each), as in a sorting line
 * that scores frames of uneven size: frame f has n[f] rows of p[f] columns,
 * row stride ld[f], coverage h[f].  The frames run concurrently on nstreams
 * streams (1 .. RTD_BATCH_MAX_STREAMS), each with its own workspace slice;
 * host threads take the frames in order from a shared counter.  The work
 * starts after everything earlier on `stream` and the call returns when every
 * frame is done.
 *   X[f]        device or host rows of frame f
 *   opt         shared by all frames; its subset_out, diag_out and profile
 *               are ignored
 *   out         nframes results (host)
 *   d2_out, flags_out  nullable arrays of nframes nullable per-frame outputs
 * Every frame is validated before any device work: RTD_EINVAL (with the
 * offending frames' out[f].status set) if any is invalid.  Otherwise returns
 * RTD_OK or the first nonzero frame status in frame order.
 */
int rtdetmcd_fit_batch(int32_t nframes, const float* const* X, const int64_t* n, const int32_t* p,
                       const int64_t* ld, const int64_t* h, const rtd_options* opt,
                       void* workspace, size_t ws_bytes, void* stream, int32_t nstreams,
                       rtd_result* out, float* const* d2_out, uint8_t* const* flags_out);

/* Bytes of workspace rtdetmcd_distances needs. */
size_t rtdetmcd_distances_workspace_size(int64_t n, int32_t p);

/*
 * Squared statistical distances d2_i = (x_i - mu)^T Sigma^-1 (x_i - mu)
 * (Section 2.1) computed as ||L^-1 (x_i - mu)||^2 with Sigma = L L^T
 * (Section 3.4): the scoring step of Section 6.
 *   mu_host     p doubles (host)
 *   sigma_host  p x p doubles, row-major (host); must be positive definite
 *               (RTD_EDEGENERATE otherwise)
 *   precision   RTD_FP32 or RTD_FP64 arithmetic for the row pass
 *   d2_out      n floats
 */
int rtdetmcd_distances(const float* X, int64_t n, int32_t p, int64_t ld,
                       const double* mu_host, const double* sigma_host,
                       int32_t precision, float* d2_out,
                       void* workspace, size_t ws_bytes, void* stream);

/* Bytes of workspace rtdetmcd_score needs. */
size_t rtdetmcd_score_workspace_size(int64_t n, int32_t p);

/*
 * Scoring of rows against a fit in one pass (Section 6: the distances and
 * flags of Section 4 step 10 for new data): d2_i = (x_i - mu)^T Sigma^-1
 * (x_i - mu) and the flag d2_i > cutoff_d2, both written by the same
 * streaming kernel, with the number of flagged rows.
 *   mu_host, sigma_host  the fit (host; sigma positive definite, else
 *                        RTD_EDEGENERATE); passed in the launch parameters,
 *                        so no copy of them precedes the stream
 *   cutoff_d2            e.g. rtdetmcd_chi2_quantile(p, 0.975)
 *   precision            RTD_FP32: FP32 rows, and a row whose FP32 d2 lies
 *                        within 2^-9 of the cutoff is decided by its FP64
 *                        distance (so the flags equal those of FP64
 *                        distances); RTD_FP64: FP64 rows
 *   d2_out               nullable, n floats
 *   flags_out            nullable, n bytes (1 = outlier)
 *   n_flagged            nullable, host: the count (-1 without flags_out)
 */
int rtdetmcd_score(const float* X, int64_t n, int32_t p, int64_t ld, const double* mu_host,
                   const double* sigma_host, double cutoff_d2, int32_t precision, float* d2_out,
                   uint8_t* flags_out, int64_t* n_flagged, void* workspace, size_t ws_bytes, void* stream);

/*
 * Scoring many batches of rows against one fit (Section 6: every image of a
 * sorting line scored with the same fit).  rtdetmcd_score_prepare factorises
 * the fit (mu, sigma as for rtdetmcd_score, row-major p x p, host memory)
 * once into `prepared`: device memory of the current device, at least
 * rtdetmcd_prepared_size() bytes, 256-byte aligned, owned by the caller.  It
 * waits for the factorisation and returns its status (RTD_EDEGENERATE when
 * sigma is not positive definite; a prepared fit in that state makes the
 * FP32 scoring pass write nothing).
 * rtdetmcd_score_prepared then scores n rows in one kernel launch on `stream`
 * and returns without waiting for it: the d2_out, flags_out and count of
 * rtdetmcd_score (d2 and flags nullable), all device memory of the current
 * device; count (nullable, needs flags_out) is one 64-bit counter to which
 * the pass adds its number of flagged rows (the caller zeroes it).  p must be
 * the prepared fit's.  Argument errors come back at once; the pass has no
 * data-dependent errors.  Calls may overlap on several streams: the prepared
 * fit is only read.
 */
size_t rtdetmcd_prepared_size(void);
int rtdetmcd_score_prepare(const double* mu_host, const double* sigma_host, int32_t p, double cutoff_d2,
                           void* prepared, void* stream);
int rtdetmcd_score_prepared(const float* X, int64_t n, int32_t p, int64_t ld, const void* prepared,
                            int32_t precision, float* d2_out, uint8_t* flags_out, unsigned long long* count,
                            void* stream);

/* Size of the fixed device array used by rtdetmcd_distances_noalloc. */
#define RTD_NOALLOC_SCRATCH_BYTES (96 * 1024)

/*
 * Scoring without allocating: the squared distances of rtdetmcd_distances,
 * for callers that cannot allocate device memory when they score (a sorting
 * line that must not wait on an allocator between frames, code that runs in
 * a fixed memory budget, or a process whose device memory is owned by
 * another component).  The paper has no counterpart; this is an interface
 * convenience.
 *   X, d2_out  device pointers on the current device (RTD_EINVAL for host
 *              memory, whose staging would need memory proportional to n, and
 *              for another device's memory)
 *   p          <= RTD_MAX_P, the largest fit the array holds (RTD_EINVAL above)
 * The working state (factorised fit, status word) lives in one file-scope
 * device array of RTD_NOALLOC_SCRATCH_BYTES that every GPU using the library
 * keeps until the process exits.  The first call on a device looks up that
 * array's device address; make that first call before capturing any stream
 * into a CUDA graph.  All calls on a device share the array and it keeps the
 * last call's contents: calls whose device work overlaps (several threads or
 * streams at the same time) race on it and must be serialised by the caller.
 * The looked-up address is kept for the life of the process: after a
 * cudaDeviceReset of that device it is stale, so do not reset a device that
 * this entry point has used.  No cudaMalloc, cudaFree or other allocation is
 * made.
 */
int rtdetmcd_distances_noalloc(const float* X, int64_t n, int32_t p, int64_t ld,
                               const double* mu_host, const double* sigma_host,
                               int32_t precision, float* d2_out, void* stream);

/*
 * Outlier flags of Section 4 step 10: flags_out[i] = (d2[i] > cutoff_d2).
 * n_flagged (nullable, host) receives the count.  workspace >= 256 bytes.
 */
int rtdetmcd_flag(const float* d2, int64_t n, double cutoff_d2,
                  uint8_t* flags_out, int64_t* n_flagged,
                  void* workspace, size_t ws_bytes, void* stream);

/* Bytes of workspace rtdetmcd_grad needs. */
size_t rtdetmcd_grad_workspace_size(int64_t n, int32_t p);

/*
 * Adjoint of the reweighting and final-distance steps (Section 4 steps 8-10)
 * with the reweighting set W held fixed.  The paper has no counterpart: the
 * set W is a discrete choice, and with it fixed the fit is a smooth function
 * of the rows, so that a caller can differentiate a loss through it.
 *   f(X) = w_logdet * log det Sigma + w_rd * sum_i RD_i
 *   mu = mean of the rows in W, Sigma = c * S_W (sample covariance of W,
 *   denominator |W| - 1), RD_i = sqrt((x_i - mu)^T Sigma^-1 (x_i - mu)) over
 *   all n rows.
 *   X           device, n rows of stride ld floats
 *   wset        device, n bytes; row i is in W when bit `wbit` of wset[i] is
 *               set (bit 1 of rtd_options.subset_out marks the fit's W)
 *   mu_host     p doubles (host): the mean of W
 *   sigma_host  p x p doubles, row-major (host): c * S_W, as rtdetmcd_fit
 *               returns it in rtd_result.mu / .sigma with c = rtd_result.c_rew;
 *               positive definite (RTD_EDEGENERATE otherwise)
 *   value_out   nullable, host: f
 *   grad_out    nullable, device, n x p floats (row-major, stride p): df/dX.
 *               Rows with RD_i = 0 take the zero subgradient of their own
 *               distance term.
 * Returns RTD_EINVAL for host X, wset or grad_out, RTD_EDEGENERATE when
 * |W| < p + 1.  Row arithmetic in FP32, sums across rows in FP64.
 */
int rtdetmcd_grad(const float* X, int64_t n, int32_t p, int64_t ld,
                  const uint8_t* wset, int32_t wbit,
                  const double* mu_host, const double* sigma_host, double c,
                  double w_logdet, double w_rd, double* value_out, float* grad_out,
                  void* workspace, size_t ws_bytes, void* stream);

/*
 * Vector-Jacobian product of the reweighted fit (Section 4 steps 8-10) with
 * the reweighting set W held fixed: for the outputs
 *   mu = mean of the rows in W (p), Sigma = c * S_W (p x p),
 *   log det Sigma, and RD_i = sqrt((x_i - mu)^T Sigma^-1 (x_i - mu)) (n rows),
 * and cotangents (gmu, gSigma, g_logdet, gRD) on them, grad_out receives
 *   d/dX [ gmu . mu + <gSigma, Sigma> + g_logdet log det Sigma + gRD . RD ].
 * The paper has no counterpart: W and the h-subsets are discrete choices,
 * and with them fixed the fit is smooth in the rows, which gives every row's
 * influence on the fit.
 *   X, wset, wbit, mu_host, sigma_host, c   as for rtdetmcd_grad
 *   gmu_host     nullable (zero), host, p doubles
 *   gsigma_host  nullable (zero), host, p x p doubles row-major (its
 *                symmetric part acts, Sigma being symmetric)
 *   grd          nullable (zero), device, n floats: cotangent on RD
 *   grad_out     device, n x p floats (row-major, stride p)
 * Workspace: rtdetmcd_grad_workspace_size(n, p) bytes.  Returns RTD_EINVAL
 * for host X, wset, grd or grad_out and non-finite cotangents,
 * RTD_EDEGENERATE when |W| < p + 1.  Rows with RD_i = 0 take the zero
 * subgradient of their own distance.  Row arithmetic in FP32, sums across
 * rows in FP64.
 */
int rtdetmcd_vjp(const float* X, int64_t n, int32_t p, int64_t ld, const uint8_t* wset, int32_t wbit,
                 const double* mu_host, const double* sigma_host, double c, const double* gmu_host,
                 const double* gsigma_host, double g_logdet, const float* grd, float* grad_out,
                 void* workspace, size_t ws_bytes, void* stream);

/* chi2_{p, q} quantile as used for the cutoff (computed by the library's own
   incomplete-gamma routines). */
double rtdetmcd_chi2_quantile(int32_t p, double q);

/* Launch shapes of a fit picked by the autotuner. */
typedef struct {
    int32_t win_rows;     /* rows per CTA, at least, of the C-step distance pass (0: the pass's own) */
    int32_t sel_ctas;     /* CTAs per chain of the one-launch window selection */
    int32_t candidates;   /* shapes timed */
    int32_t reserved;
    double  ms_best;      /* median fit time under the chosen shape */
    double  ms_default;   /* median fit time under the default shape */
} rtd_tuning;

/*
 * Autotuner of the launch shapes (a part of this engine, not of the paper):
 * times whole fits of these rows (one warm-up and three timed fits per
 * candidate, CUDA events on `stream`) under each candidate shape of the
 * C-step distance pass (rows per CTA) and of the window selection (CTAs per
 * chain), and keeps the fastest for later fits with the same padded width,
 * block count, block length class, form and paths, in this process.  Neither
 * shape changes any value a fit computes, so tuned and untuned fits are
 * equal bit for bit.  Arguments as for rtdetmcd_fit (device rows; the fits'
 * outputs are not kept); `out` (nullable, host) receives the choice.
 */
int rtdetmcd_autotune(const float* X, int64_t n, int32_t p, int64_t ld, int64_t h, const rtd_options* opt,
                      void* workspace, size_t ws_bytes, void* stream, rtd_tuning* out);

/* The tuned shape for fits of this size and these options: 1 and *out filled
   if one is kept, 0 otherwise. */
int rtdetmcd_tuned(int64_t n, int32_t p, const rtd_options* opt, rtd_tuning* out);

/* Human-readable name of a status code. */
const char* rtdetmcd_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* RTDETMCD_H */
