/*
 * ig.h -- C ABI of the GB300 (sm_103a) Interpretable Generalization library.
 *
 * Interpretable Generalization (IG) learns, from labelled records encoded as
 * itemsets, the "coherent" patterns of each class -- itemsets that occur in
 * records of one class and inside no record of the other -- and scores new
 * records by the patterns they contain (paper Section 3.1, Eq. 1-4 and
 * Regulations 1-3; packed layout Eq. 5; subset test Eq. 6).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  * Records are itemsets over L items, bit-packed into K = ceil(L/64) 64-bit
 *    words (Eq. 5): item j is bit (j mod 64) of word (j div 64).  Bits at
 *    positions >= L must be zero: a set tail bit counts as an item.  A record
 *    matrix is row-major uint64[n][K].  1 <= K <= IG_MAX_WORDS.
 *  * Classes: label 1 = attack (class "+", evidence A), 0 = normal (class
 *    "-", evidence N).
 *  * Pattern lists are in canonical order: ascending as K-word unsigned
 *    integers, word K-1 most significant; no duplicates; no empty pattern.
 *  * Array arguments may be device pointers (CUDA memory of the current
 *    device) or host pointers (pageable or pinned); the library detects which
 *    with cudaPointerGetAttributes.  Host inputs are copied to the device and
 *    host outputs copied back inside the call, which then returns only after
 *    the copy-back has completed.  With device pointers all work is enqueued
 *    on `stream` and the call may return before it has finished, except where
 *    a size must be known on the host (noted per function).
 *  * The caller owns every array it passes.  Arrays of data-dependent size
 *    (pattern lists) belong to the library's ig_model and live until
 *    ig_model_free.
 *  * Every function returns IG_OK (0) or a negative status; the calling
 *    thread's last error message is then readable via ig_last_error().  No
 *    C++ exception leaves the library: a failed host allocation inside a
 *    call is reported as IG_E_NOMEM, any other exception as IG_E_INTERNAL.
 *    There is no CPU fallback: without a usable GPU every compute call
 *    returns IG_E_CUDA.
 */
#ifndef IG_GB300_H
#define IG_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same object as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st* ig_stream_t;

enum {
  IG_OK = 0,
  IG_E_INVAL = -1,     /* bad argument (size, K, label or code out of range) */
  IG_E_NOMEM = -2,     /* device or host allocation failed */
  IG_E_CUDA = -3,      /* CUDA runtime error (message has the CUDA text) */
  IG_E_TIMEOUT = -4,   /* a bounded device-side wait ran out */
  IG_E_OVERFLOW = -5,  /* a count exceeded the library's index range */
  IG_E_INTERNAL = -6,  /* internal consistency check failed */
  IG_E_IO = -7         /* file could not be read or written */
};

#define IG_MAX_WORDS 16 /* K limit: itemsets of up to 1024 items */

/* Fitted model: the coherent dictionaries P+ and P- with their supports and
 * scores, plus the Regulation 3 statistics.  Opaque; device-resident. */
typedef struct ig_model ig_model;

typedef struct {
  /* Regulation 3 (Section 3.1): when reg3_enabled != 0, a record whose
   * normal evidence N < mu_N - r * sigma_N is labelled attack even where
   * Regulation 1 says normal.  mu_N and sigma_N are the mean and population
   * standard deviation of N over the training normal records, computed in
   * double precision in record order. */
  double r;
  int32_t reg3_enabled;
  /* Subset-test form: 0 = library default (4 where K rounds up to 2, 4 or
   * 8; 3 where it rounds up to 16; 1 for K = 1);
   * 1 = integer-pipe kernel (LOP3) on every pair; 2 = tensor-core kernel
   * (tcgen05 0/1 GEMM) on every pair, where K (rounded up to a power of two)
   * is 2, 4 or 8, else 1; 3 = item index: each pattern is tested only
   * against the records holding its rarest item (exact), in integer-pipe
   * blocks, falling back to 2 when records are too dense for the index to
   * pay off; 4 = item index with its blocks run as tcgen05 0/1 GEMMs (K
   * rounded up to 2, 4 or 8; else as 3).  The choice is kept in the model
   * and used by ig_score too.  Results are identical for every choice. */
  int32_t subset_kernel;
  /* Tiling of the item-index form (results never depend on them; 0 picks
   * the default): the most own rows per thread of a block (1, 2 or 4, i.e.
   * blocks of up to 256, 512 or 1,024 rows; default 4), and the factor by
   * which one side of an item group must outnumber the other before that
   * side is held in registers instead of the result side (default 2). */
  int32_t index_max_q;
  int32_t index_flip_factor;
} ig_params;

typedef struct {
  int32_t K;                 /* words per pattern */
  int32_t reg3_enabled;
  int64_t n_train[2];        /* training records per class [normal, attack] */
  int64_t n_candidates[2];   /* |B^c|: distinct non-empty candidates (Eq. 1) */
  int64_t n_patterns[2];     /* |P^c|: coherent patterns (Eq. 3) */
  int64_t n_pairs[2];        /* intersections formed: n_c (n_c - 1) / 2 */
  double reg3_mu, reg3_sigma, reg3_r, reg3_threshold;
  int64_t coherence_tests[2];  /* subset tests the coherence step executed */
  int64_t coherence_tests_tc[2]; /* ... of which on the tensor cores */
  int64_t coherence_tests_idx[2]; /* ... of which through the item index */
  int64_t support_tests[2];      /* subset tests the support step executed */
  int32_t subset_kernel;       /* form in use: 1 integer pipe, 2 tensor cores, 3 item index,
                                  4 item index on the tensor cores */
  int32_t reserved;
} ig_model_info_t;

/* Section 3.1 / Eq. 5: one-hot encoding of discretised records.
 * codes: uint16[n][F], codes[i][f] < cards[f] (bin of feature f), or
 *        0xFFFF for a missing value (no item for that feature).
 * cards: HOST array uint16[F], feature cardinalities; item of (f, v) is
 *        sum(cards[0..f-1]) + v, so L = sum(cards).
 * words_out: uint64[n][K] with K = ceil(L/64) (the K argument must equal it).
 * Returns IG_E_INVAL if a code is out of range (checked on the device; the
 * call synchronizes `stream` to read the check). n == 0 is valid. */
int ig_encode(const uint16_t* codes, int64_t n, int32_t F,
              const uint16_t* cards, uint64_t* words_out, int32_t K,
              ig_stream_t stream);

/* IG training (Section 3.1): for each class c, the candidates B^c of Eq. 1
 * (pairwise intersections of class-c records plus the records themselves,
 * as a set, the empty itemset dropped), the coherent subset P^c of Eq. 3
 * (no record of the other class contains the pattern, tested as in Eq. 6),
 * and for each coherent pattern its support f_c (number of class-c records
 * containing it, duplicates counted) and score S_c = f_c * |b|^2 (Eq. 2),
 * |b| = number of items.
 * rows: uint64[n][K]; labels: uint8[n] in {0, 1}.  Both classes must be
 * non-empty (IG_E_INVAL otherwise).  p may be NULL (defaults: Regulation 3
 * off).  On success *out receives a new model (free with ig_model_free).
 * Synchronizes `stream` at internal size checkpoints; returns after the
 * model is complete. */
int ig_fit(const uint64_t* rows, const uint8_t* labels, int64_t n, int32_t K,
           const ig_params* p, ig_model** out, ig_stream_t stream);

/* One problem of a batched fit: records and labels as for ig_fit. */
typedef struct {
  const uint64_t* rows;   /* uint64[n][K], device or host */
  const uint8_t* labels;  /* uint8[n] */
  int64_t n;
  int32_t K;
  int32_t reserved;
  const ig_params* params; /* this problem's parameters, or NULL for the batch's */
} ig_problem;

/* Batched IG training: fits n_problems independent problems (each exactly
 * as ig_fit would, Section 3.1), of any sizes and word counts.  The
 * candidate stage (Eq. 1) of every class of every problem runs first, in one
 * launch of a persistent kernel whose blocks draw (problem, class, pair
 * tile) work from a device-side queue (further launches only for tables
 * that run out of room).  The remaining steps of each fit then run
 * concurrently on up to `lanes` streams (0 = 8); the largest problems start
 * first and every lane pulls the next problem when it finishes one.  The
 * batch-level scheduling of Section 3.3 (batch size as a tunable parameter)
 * applied across independent problems.  out[i] receives
 * problem i's model.  Work is ordered after what `stream` holds when the
 * call starts and before what is enqueued on it afterwards; the call returns
 * when all models are complete.  On an error every model is freed, out[] is
 * cleared, and the first error is reported (naming the problem). */
int ig_fit_batched(const ig_problem* problems, int32_t n_problems, const ig_params* p,
                   int32_t lanes, ig_model** out, ig_stream_t stream);

/* One job of a batched scoring call: records of the model's width K and
 * the outputs, exactly as for ig_score. */
typedef struct {
  const ig_model* model;
  const uint64_t* rows;  /* uint64[m][K], device or host */
  int64_t m;
  int64_t* A_out;        /* int64[m], device or host */
  int64_t* N_out;        /* int64[m] */
  uint8_t* label_out;    /* uint8[m] */
} ig_score_job;

/* Batched IG inference: n_jobs independent scoring calls (evidence of Eq. 4
 * and the labels of Regulations 1-3, each exactly as ig_score computes it;
 * jobs may share a model) run concurrently on up to `lanes` streams (0 = 8),
 * the largest batches first, every lane pulling the next job when it
 * finishes one -- the batch-level scheduling of Section 3.3 applied across
 * independent problems.  Work is ordered after what `stream` holds when the
 * call starts and before what is enqueued on it afterwards; the call
 * returns when every result is in place.  On an error the first error is
 * reported (naming the job); the other jobs' outputs are then unspecified. */
int ig_score_batched(const ig_score_job* jobs, int32_t n_jobs, int32_t lanes,
                     ig_stream_t stream);

/* Builds a model from given pattern sets (Section 3.1's dictionaries P^-
 * and P^+, learned elsewhere), e.g. to serve them: for class c (0 = normal,
 * 1 = attack) words[c] is uint64[n_patterns[c]][K] (any order; non-empty,
 * distinct rows) and support[c] uint32[n_patterns[c]] the supports f_c.  The
 * model holds the patterns in canonical order with their supports and the
 * scores S = f * |b|^2 of Eq. 2; Regulation 3 is off.  IG_E_INVAL for an
 * empty or repeated pattern.  Returns when the model is complete. */
int ig_model_from_patterns(int32_t K, const uint64_t* const* words, const uint32_t* const* support,
                           const int64_t* n_patterns, ig_model** out, ig_stream_t stream);

/* Sizes and statistics of a fitted model (see ig_model_info_t): per class
 * the training records, |B^c| (Eq. 1), |P^c| (Eq. 3) and the subset tests
 * executed, plus Regulation 3's mu_N, sigma_N, r and threshold.  Host only;
 * IG_E_INVAL if m or info is NULL. */
int ig_model_info(const ig_model* m, ig_model_info_t* info);

/* Device pointers to class `cls` (1 = attack P+, 0 = normal P-) of a model,
 * the dictionary of Section 3.1 (coherent patterns, Eq. 3) with the supports
 * f_c and scores S_c of Eq. 2: words uint64[n_patterns][K] in canonical
 * order, support uint32[n_patterns], score uint64[n_patterns].  Any output
 * pointer may be NULL.  The arrays are owned by the model and live until
 * ig_model_free.  IG_E_INVAL for a NULL model or cls not 0 or 1. */
int ig_model_patterns(const ig_model* m, int32_t cls, const uint64_t** words,
                      const uint32_t** support, const uint64_t** score);

/* Copies class `cls` of a model (its patterns, Eq. 3, with f_c and S_c of
 * Eq. 2) into caller arrays (device or host; any may be NULL): words_out
 * uint64[n_patterns][K], support_out uint32[n_patterns], score_out
 * uint64[n_patterns].  Returns after the copies have completed.  IG_E_INVAL
 * for a NULL model or cls not 0 or 1; IG_E_CUDA if a copy fails. */
int ig_model_copy_patterns(const ig_model* m, int32_t cls, uint64_t* words_out,
                           uint32_t* support_out, uint64_t* score_out,
                           ig_stream_t stream);

/* IG inference (Eq. 4 and Regulations 1-3): for each record x,
 * A(x) = sum of S+(b) over b in P+ contained in x, N(x) likewise over P-,
 * both exact int64; label = 1 (attack) if A >= N (Regulation 1), or
 * A == N == 0 (Regulation 2), or Regulation 3 fires; else 0.
 * rows: uint64[m][K] with the model's K.  A_out, N_out: int64[m];
 * label_out: uint8[m]; any of the three may be NULL.  m == 0 is valid. */
int ig_score(const ig_model* model, const uint64_t* rows, int64_t m,
             int64_t* A_out, int64_t* N_out, uint8_t* label_out,
             ig_stream_t stream);

/* Scoring that allocates no device memory (the paper has no counterpart:
 * this is a library convenience).  It is for callers that cannot have the
 * library allocate on their behalf -- a latency-bound flow-scoring loop where
 * a cudaMalloc/cudaFree could stall the device or fail under memory pressure,
 * or a process whose device memory is reserved up front by another
 * allocator.  Results equal ig_score's.
 * rows, and each non-NULL output, must be device memory; at most
 * IG_SCORE_NOALLOC_MAX_ROWS rows per call (IG_E_INVAL beyond that, and for
 * host pointers).  The A/N accumulators and the status word live in one
 * fixed device array inside the library (about 4 MiB, held on every GPU that
 * loads the library until the process exits); it is cleared by each call, and
 * calls whose work overlaps on the GPU race on it.  The first call on each
 * device looks up that array's device address.  Synchronizes `stream` before
 * returning (to read the status word), so a call cannot be captured into a
 * CUDA graph. */
#define IG_SCORE_NOALLOC_MAX_ROWS 262144
int ig_score_noalloc(const ig_model* model, const uint64_t* rows, int64_t m,
                     int64_t* A_out, int64_t* N_out, uint8_t* label_out,
                     ig_stream_t stream);

/* ---- Serving ------------------------------------------------------------
 * A scoring server over a device-resident model (Eq. 4 and Regulations 1-3
 * per flow, exactly as ig_score; the paper has no serving layer -- it notes
 * that per-flow inference on learned patterns takes milliseconds).
 * Requests are host arrays of packed flows.  The server batches the requests
 * waiting in its queue -- in arrival order, as many as fit max_batch_flows
 * and the device-memory budget for work in flight, without waiting for more
 * -- and runs up to `slots` batches at once on separate streams, so batches
 * admitted while others run overlap on the device.  A flow's results do not
 * depend on the batch it shares. */
typedef struct ig_server ig_server;
typedef struct {
  int32_t slots;                /* batches in flight at once (0 = 3) */
  int32_t reserved;
  int64_t max_batch_flows;      /* flows per batch, and per request (0 = 65536) */
  int64_t memory_budget_bytes;  /* device bytes for batches in flight (0 = a
                                   quarter of the free memory at creation) */
} ig_server_config;

/* Continuous-batching scoring server: the inference of Section 3.3 (the
 * evidence of Eq. 4 and the labels of Regulations 1-3, exactly as ig_score)
 * served per flow as the abstract sets out.  Requests that arrive while
 * others run are admitted into batches as slots and the memory budget allow;
 * admitted batches run concurrently, one stream per slot, and every flow's
 * result equals ig_score's.  The model must outlive the server.  cfg may be
 * NULL.  IG_E_INVAL for a NULL model or out; IG_E_NOMEM if its device or
 * pinned buffers cannot be allocated. */
int ig_server_create(const ig_model* model, const ig_server_config* cfg, ig_server** out);
/* Queues a request: rows uint64[m][K] on the host (read when the request is
 * batched), results written to the host arrays A_out, N_out (int64[m]) and
 * label_out (uint8[m]; any may be NULL) before the request completes.  The
 * arrays must stay valid until ig_server_wait returns for *ticket.
 * IG_E_INVAL for a NULL server, rows or ticket, m <= 0, or m above the
 * batch cap. */
int ig_server_submit(ig_server* sv, const uint64_t* rows, int64_t m, int64_t* A_out,
                     int64_t* N_out, uint8_t* label_out, uint64_t* ticket);
/* Blocks until the request completes; *latency_ms (may be NULL) receives the
 * time from its submission to its completion.  Each ticket is waited once.
 * Returns the request's own status (a scoring error is reported here), or
 * IG_E_INVAL for a NULL server or an unknown ticket. */
int ig_server_wait(ig_server* sv, uint64_t ticket, double* latency_ms);
/* Batches run and flows scored so far.  IG_E_INVAL for a NULL server. */
int ig_server_stats(ig_server* sv, int64_t* batches, int64_t* flows);
/* Stops the server after the batches in flight; requests still queued are
 * dropped (destroy only once every submitted request has been waited). */
void ig_server_destroy(ig_server* sv);

/* Model persistence (no counterpart in the paper): a flat little-endian file
 * (magic, version, K, counts, Regulation 3 statistics, then per class the
 * canonical words, supports and scores of Eq. 2).  ig_model_load places the
 * model on the current device.  Errors: IG_E_INVAL for NULL arguments;
 * IG_E_IO for a file that cannot be opened or written, has another magic,
 * version or K out of range, or whose pattern counts do not account for its
 * size exactly (checked before anything is allocated); IG_E_CUDA for a
 * failed device allocation or copy. */
int ig_model_save(const ig_model* m, const char* path);
int ig_model_load(const char* path, ig_model** out);
void ig_model_free(ig_model* m);

/* Message for the calling thread's most recent failed call ("" if none). */
const char* ig_last_error(void);

/* Per-stage device timing.  While enabled, the library records CUDA events
 * around every kernel launch on the launching stream; ig_prof_read
 * synchronizes and returns, for each stage s < IG_PROF_STAGES, the summed
 * kernel time in milliseconds and the number of launches since the last
 * reset.  Stage names are given by ig_prof_stage_name. */
#define IG_PROF_STAGES 20
int ig_prof_enable(int32_t on);
/* Times only the stages s with bit s of stage_mask set (all stages until
 * the first call); the others launch without events.  Executed-test counts
 * (ig_prof_read_work) are kept for every stage while enabled.  Lets a
 * caller time one stage without the cost of events around all the others. */
int ig_prof_select(uint32_t stage_mask);
int ig_prof_reset(void);
int ig_prof_read(double* ms, int64_t* launches);
const char* ig_prof_stage_name(int32_t stage);

/* Instrumentation (no counterpart in the paper).  Timeline of the stages
 * recorded since the last reset (which also records
 * the reference point): for each of the first min(cap, *n_out) stage spans,
 * its stage id, the stream it ran on (an opaque id), and its begin and end
 * in milliseconds after the reset.  Synchronizes the recorded events.  Any
 * output array may be NULL; *n_out receives the number of spans. */
int ig_prof_timeline(int32_t* stage, uint64_t* stream, double* t0_ms, double* t1_ms,
                     int64_t cap, int64_t* n_out);

/* Subset tests executed per stage since the last reset, counted while
 * timing is enabled (support and evidence stages; coherence tests are
 * reported per model by ig_model_info). */
int ig_prof_read_work(int64_t* tests);

/* Number of kernels this library has launched in the process so far. */
int64_t ig_launch_count(void);

/* ---- Throughput probes --------------------------------------------------
 * Measured rates of the hardware units the kernels above are bound by, for
 * roofline denominators (instrumentation: the paper has no counterpart).
 *   IG_PROBE_LOP3       LOP3 (three-input 32-bit logic) instructions per
 *                       second over all SMs -- the integer-pipe subset test
 *                       (Eq. 6 as acc |= p & ~r) takes one per half word;
 *   IG_PROBE_L2_READ    bytes per second of coalesced 16-byte loads over a
 *                       buffer of `arg` MiB (0 = 48) that stays in L2;
 *   IG_PROBE_L2_RANDOM  bytes per second of 16-byte loads at random 16-byte
 *                       offsets of such a buffer (the dedup table's access);
 *   IG_PROBE_MMA_F8_SMEM, IG_PROBE_MMA_F8_TMEM
 *                       flops per second of back-to-back tcgen05.mma
 *                       kind::f8f6f4 chains (E4M3 operands, FP32
 *                       accumulators), M = 128, N = arg & 0xfff (64, 128,
 *                       or 256 with A in shared memory only), 16 MMAs of
 *                       K = 32 per chain, A read from shared or tensor
 *                       memory; one CTA per SM.  arg bit 12: a commit after
 *                       every chain; bit 13: chains alternate between two
 *                       accumulators and chain c waits for chain c - 2 to
 *                       complete (an accumulator ring of two).
 * A warm-up launch precedes the timed one.  *rate receives the rate, *ms the
 * timed launch's device time, *cycles (MMA probes) the largest SM-clock count
 * a CTA spent issuing and draining its chains; any may be NULL.  Runs on the
 * current device on a stream of its own and synchronizes it.  IG_E_INVAL for
 * an unknown probe or shape. */
enum {
  IG_PROBE_LOP3 = 0,
  IG_PROBE_L2_READ = 1,
  IG_PROBE_L2_RANDOM = 2,
  IG_PROBE_MMA_F8_SMEM = 3,
  IG_PROBE_MMA_F8_TMEM = 4
};
int ig_probe(int32_t probe, int32_t arg, double* rate, double* ms, double* cycles);

#ifdef __cplusplus
}
#endif
#endif /* IG_GB300_H */
