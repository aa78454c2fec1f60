/*
 * spdz.h -- C ABI of the B300 (sm_103a) SPDZ online-phase library.
 *
 * The library evaluates the online phase of SPDZ (An LLVM-Based Optimization
 * Pipeline for SPDZ, arXiv 2512.11112, Sec. II-A) on additively secret-shared,
 * MAC-authenticated field elements.  All n parties are simulated on one GPU:
 * each party's value shares and MAC shares are separate device rows, so
 * opening a value is an on-device sum over the party rows.
 *
 * Fields: p = 2^61 - 1 (one uint64 per element), p = 2^127 - 1 (two uint64
 * words per element, low word first, 16-byte aligned) and p = 2^32 - 5, the
 * prime of the paper's evaluation (Sec. IV-A; one uint32 per element).  Host
 * constants passed to the calls use the same element formats.  Every stored
 * share is canonical, in [0, p).  All arithmetic is exact; nothing here
 * changes the protocol's results.  Circuits, the tagged plan and matrix
 * products name the fields they accept.
 *
 * Conventions for every call:
 *   - Returns an int status (SPDZ_OK or one of the SPDZ_ERR_* codes below);
 *     no call aborts the process or traps the device.  spdz_last_error()
 *     returns a text description of the last failure on the context.
 *   - Device pointers are owned by the caller (for example torch tensors);
 *     the library never frees them.  Host pointers are read or written
 *     during the call only.
 *   - Work is enqueued on the context's stream, in call order.  Calls that
 *     return a result to the host (spdz_mac_check, spdz_run_dag with stats)
 *     synchronise that stream.  A context is not thread-safe.
 */
#ifndef SPDZ_H
#define SPDZ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ codes */
enum spdz_status {
    SPDZ_OK = 0,
    SPDZ_ERR_ARG = 1,      /* bad argument (null pointer, size, field, op) */
    SPDZ_ERR_ALIGN = 2,    /* a device pointer or stride breaks the alignment rule */
    SPDZ_ERR_OOM = 3,      /* device allocation failed or budget exceeded */
    SPDZ_ERR_TRIPLES = 4,  /* not enough unused triples: a triple is never reused (Sec. II-A.3) */
    SPDZ_ERR_MAC = 5,      /* MAC check failed: the protocol aborts (Sec. II-A.4) */
    SPDZ_ERR_TIMEOUT = 6,  /* a bounded device wait gave up; the results are invalid */
    SPDZ_ERR_CUDA = 7,     /* a CUDA runtime call failed */
    SPDZ_ERR_STATE = 8     /* call not valid in the context's current state */
};

enum spdz_field { SPDZ_F61 = 0, SPDZ_F127 = 1, SPDZ_F32 = 2 };

/* Gate / linear-operation codes (Sec. II-A.3 addition; Sec. III-B gate set:
 * shl by k lowers to a public-constant multiply by 2^k). */
enum spdz_op {
    SPDZ_OP_ADD = 0,   /* z = x + y                                     */
    SPDZ_OP_SUB = 1,   /* z = x - y                                     */
    SPDZ_OP_CMUL = 2,  /* z = k * x, k public                           */
    SPDZ_OP_CADD = 3,  /* z = x + k, k public                           */
    SPDZ_OP_MUL = 4    /* z = x * y by a Beaver triple (circuits only)  */
};

/* Dealer array kinds: the stream-id "kind" field of the counter PRG. */
enum spdz_kind {
    SPDZ_KIND_ALPHA = 1, SPDZ_KIND_TRIPLE_A = 2, SPDZ_KIND_TRIPLE_B = 3,
    SPDZ_KIND_TRIPLE_C = 4, SPDZ_KIND_INPUT = 5, SPDZ_KIND_CHECK = 6,
    SPDZ_KIND_MTRIPLE_A = 7, SPDZ_KIND_MTRIPLE_B = 8, SPDZ_KIND_MTRIPLE_C = 9,
    SPDZ_KIND_INPUT_MASK = 10  /* masks of private inputs; stream sub = the owning party */
};

#define SPDZ_MAX_PARTIES 8

/* A secret-shared array on the device (Sec. II-A.2: party i holds (x_i, m_i)).
 * Party i's value shares start at val + i*stride elements and its MAC shares
 * at mac + i*stride elements.  A view of elements [off, off+len) is the same
 * struct with both pointers advanced by off elements.  Pointers must be
 * 8-byte aligned (16-byte for p127); 16-byte alignment of the rows enables
 * 128-bit vector access for p61. */
typedef struct {
    void *val;
    void *mac;
    int64_t stride;
} spdz_buf;

typedef struct spdz_ctx spdz_ctx;

/* ---------------------------------------------------------------- context
 * Creates a context for n_parties (2..SPDZ_MAX_PARTIES) parties over `field`,
 * enqueuing on `stream` (a cudaStream_t; NULL = legacy default stream) of the
 * current device.  The context owns a small device workspace (MAC-check
 * accumulators, the epoch key, barrier counters) and nothing else.
 * Errors: SPDZ_ERR_ARG, SPDZ_ERR_CUDA, SPDZ_ERR_OOM. */
int spdz_ctx_create(spdz_ctx **out, int n_parties, int field, void *stream);
int spdz_ctx_destroy(spdz_ctx *ctx);
const char *spdz_last_error(const spdz_ctx *ctx);
/* Replaces the context's stream (for example torch's current stream). */
int spdz_ctx_set_stream(spdz_ctx *ctx, void *stream);

/* ------------------------------------------------------- preprocessing
 * Dealer ("fake preprocessing", Sec. IV-A) on the device.  Elements follow the
 * counter-PRG specification (SplitMix64 counter form; stream id = kind<<56 |
 * role<<48 | party<<40 | sub), so the CPU reference can regenerate any element
 * by index.
 *
 * spdz_deal_alpha: writes the n shares of the MAC key alpha (Sec. II-A.2) to
 *   alpha_shares_dev ([n] elements, device).
 * spdz_deal_shared: elements j0 .. j0+count-1 of the shared array (kind, sub):
 *   secret uniform (or, when secret_dev is non-NULL, read from it), value and
 *   MAC shares written to `out`; alpha_shares_dev are the shares it MACs under.
 *   If secret_out_dev is non-NULL the secrets are also written there.
 * spdz_deal_triples: Beaver triples j0 .. j0+count-1 (a, b uniform, c = a*b,
 *   Sec. II-A.3) with MACs, written to a, b, c.
 * Errors: SPDZ_ERR_ARG, SPDZ_ERR_ALIGN, SPDZ_ERR_CUDA. */
int spdz_deal_alpha(spdz_ctx *ctx, uint64_t seed, void *alpha_shares_dev);
int spdz_deal_shared(spdz_ctx *ctx, uint64_t seed, uint32_t kind, uint64_t sub, uint64_t j0,
                     int64_t count, const void *alpha_shares_dev, const void *secret_dev,
                     const spdz_buf *out, void *secret_out_dev);
int spdz_deal_triples(spdz_ctx *ctx, uint64_t seed, uint64_t j0, int64_t count,
                      const void *alpha_shares_dev, const spdz_buf *a, const spdz_buf *b,
                      const spdz_buf *c);

/* Registers the preprocessing the online phase consumes: the n alpha shares
 * (copied into the context) and a pool of n_triples Beaver triples (a, b, c
 * with MACs, Sec. II-A.3), which is referenced, not copied.  Triples are
 * consumed in order by a cursor; a triple is never handed out twice
 * (SPDZ_ERR_TRIPLES when the pool runs out).  Resets the cursor to 0. */
int spdz_load_preproc(spdz_ctx *ctx, const void *alpha_shares_dev, const spdz_buf *a,
                      const spdz_buf *b, const spdz_buf *c, int64_t n_triples);
/* Number of unused triples left in the pool. */
int spdz_triples_left(const spdz_ctx *ctx, int64_t *left);

/* --------------------------------------------------------- online phase */

/* Local linear gate over N elements (Sec. II-A.3, Addition): ADD/SUB add or
 * subtract value and MAC shares; CMUL multiplies both by the public k; CADD
 * adds k to party 0's value share and alpha_i*k to every MAC share.  k_host
 * points to one field element in host memory (ignored for ADD/SUB); y may be
 * NULL for CMUL/CADD.  z may alias x or y element for element.
 * Errors: SPDZ_ERR_ARG, SPDZ_ERR_ALIGN, SPDZ_ERR_STATE (CADD before alpha is
 * loaded), SPDZ_ERR_CUDA. */
int spdz_linear(spdz_ctx *ctx, int op, const spdz_buf *x, const spdz_buf *y,
                const void *k_host, const spdz_buf *z, int64_t N);

/* Beaver multiplication of N element pairs (Sec. II-A.3, Multiplication):
 * consumes the next N triples; each party masks eps_i = x_i - a_i and
 * delta_i = y_i - b_i, the values are opened by summing over parties, and
 *   z_i = c_i + eps*b_i + delta*a_i + [i == 0] eps*delta
 *   gamma(z)_i = gamma(c)_i + eps*gamma(b)_i + delta*gamma(a)_i + alpha_i*eps*delta.
 * The opened values join the current MAC-check epoch (eps_j then delta_j);
 * their random-linear-combination terms are accumulated in the same pass.
 * If opened_dev is non-NULL it receives the public values, [2N] elements,
 * eps_j at 2j and delta_j at 2j+1.  z must not alias x, y or the triples.
 * Errors: SPDZ_ERR_ARG, SPDZ_ERR_ALIGN, SPDZ_ERR_TRIPLES, SPDZ_ERR_STATE,
 * SPDZ_ERR_CUDA. */
int spdz_mul_batch(spdz_ctx *ctx, const spdz_buf *x, const spdz_buf *y, const spdz_buf *z,
                   int64_t N, void *opened_dev);

/* Opens N shared values (Sec. II-A.3): out_dev[j] = sum_i x_i[j] ([N]
 * elements, device).  The values and their MAC shares join the current
 * MAC-check epoch. */
int spdz_open(spdz_ctx *ctx, const spdz_buf *x, void *out_dev, int64_t N);

/* Sets the seed of the MAC-check coefficients and restarts the epoch count at
 * 0.  The coefficient of the j-th value opened in epoch e is element j of the
 * PRG stream (SPDZ_KIND_CHECK, 0, 0, e) under this seed.  Must be called with
 * no value opened since the last check (SPDZ_ERR_STATE otherwise). */
int spdz_set_check_seed(spdz_ctx *ctx, uint64_t seed);

/* Batched MAC check (Sec. II-A.2/II-A.4, III-D.3) over every value opened in
 * the current epoch: A = sum r_j v_j, S_i = sum r_j gamma_i(v_j),
 * sigma_i = S_i - alpha_i*A; passes iff sum_i sigma_i == 0.  Writes *passed
 * (1/0) and, if sigma_host is non-NULL, the n sigma_i (host, [n] elements);
 * then starts the next epoch.  Synchronises the stream.  Returns SPDZ_ERR_MAC
 * when the check fails (the caller must abort the computation). */
int spdz_mac_check(spdz_ctx *ctx, int *passed, void *sigma_host);
/* Number of values opened in the current epoch, and the epoch number. */
int spdz_check_state(const spdz_ctx *ctx, int64_t *opened, int64_t *epoch);

/* `count` secret-shared inner products of length `len` (ReduceAdd over a
 * MultBatch, Sec. III-B): terms x[t*len + k], y[t*len + k]; each term is a
 * Beaver product (consuming count*len triples and opening its eps, delta in
 * one batch); the products' shares are summed locally into z[t] (value and
 * MAC), with no further open. */
int spdz_innerprod_batch(spdz_ctx *ctx, const spdz_buf *x, const spdz_buf *y,
                         const spdz_buf *z, int64_t count, int64_t len);

/* Public elementwise field arithmetic on device arrays: out[j] = a[j] op b[j]
 * for op in {ADD, SUB, CMUL (= multiply)}.  Exposes the library's modular
 * arithmetic so it can be checked against exact integer arithmetic. */
int spdz_field_op(spdz_ctx *ctx, int op, const void *a_dev, const void *b_dev, void *out_dev,
                  int64_t N);


/* ------------------------------------------------------------- circuits
 * A straight-line arithmetic circuit whose independent gates are already
 * grouped into layers (the batched regions of Sec. III-B/III-C): gate g of
 * layer l reads wires in0[g], in1[g] written by earlier layers (or inputs)
 * and writes wire n_inputs + g.  The t-th MUL gate in gate order consumes
 * the t-th triple of the run and opens eps_t, delta_t at check-log indices
 * 2t, 2t+1; a run is one MAC-check epoch of its own. */
#define SPDZ_MAX_GROUPS 256

typedef struct {
    int64_t n_inputs;              /* input wires 0 .. n_inputs-1 */
    int64_t n_gates;
    int32_t depth;                 /* number of layers */
    const int64_t *layer_offsets;  /* host [depth+1]; layer l = gates [off[l], off[l+1]) */
    const uint8_t *ops;            /* host [n_gates] spdz_op codes */
    const uint32_t *in0;           /* host [n_gates] first operand wire */
    const uint32_t *in1;           /* host [n_gates] second operand wire (ignored by CMUL/CADD) */
    const void *kconst;            /* host [n_gates] elements: constant of CMUL/CADD gates */
} spdz_dag_desc;

typedef struct spdz_dag spdz_dag;

enum spdz_sched {
    SPDZ_SCHED_PER_LAYER = 0,  /* one kernel launch per layer and gate class (MUL, linear) */
    SPDZ_SCHED_FUSED = 1,      /* persistent kernel per layer group, device barriers between layers */
    SPDZ_SCHED_TAGGED = 2      /* p = 2^61-1 only: one persistent kernel like FUSED (one group),
                                  over a tagged copy of the wires.  Every share below 2^61 leaves
                                  the top three bits of its 64-bit word free: gates also write
                                  their outputs to a wire-major copy of the wires (owned by the
                                  circuit, (n_inputs + n_gates) x 2n words: one wire's shares of
                                  every party side by side) with a per-run tag in those bits,
                                  and read their operands from it, accepting an operand once
                                  every word carries the run's tag (an aligned 8-byte store is
                                  seen whole or not at all).  The layer barrier therefore needs
                                  no fence.  The copy is zeroed every 7 runs of the circuit so no
                                  stale word carries a current tag.  Plan fields used: block,
                                  ctas_per_sm, use_graph, spin_limit_us (bound of one barrier or
                                  operand wait), poll_ns, record_layer_times, barrier_slack
                                  and test_unwritten_tag; n_groups and barrier_extra_arrivals
                                  must be 0. */
};

/* Execution plan of a circuit run.  No plan changes any result bit. */
typedef struct {
    int32_t mode;                          /* spdz_sched */
    int32_t block;                         /* threads per CTA; 0 = 256 */
    int32_t ctas_per_sm;                   /* resident CTAs per SM (fused); 0 = as many as fit */
    int32_t use_graph;                     /* capture the run once as a CUDA graph, replay after */
    int32_t n_groups;                      /* fused: layer groups (one launch each); 0 = one group */
    int32_t group_end[SPDZ_MAX_GROUPS];    /* exclusive end layer of each group, increasing, last = depth */
    uint8_t group_flush[SPDZ_MAX_GROUPS];  /* 1: partial MAC check after the group (early abort) */
    int32_t group_ctas_per_sm[SPDZ_MAX_GROUPS]; /* per-group override of ctas_per_sm; 0 = plan value */
    int32_t record_layer_times;            /* keep per-layer device times (spdz_dag_layer_times) */
    uint32_t spin_limit_us;                /* bound of one device barrier wait; 0 = 200000 */
    int32_t barrier_extra_arrivals;        /* testing: every barrier also waits for this many
                                              arrivals that never come, so the bounded wait
                                              runs out (SPDZ_ERR_TIMEOUT); 0 in normal use */
    int32_t group_cluster[SPDZ_MAX_GROUPS];/* fused: 0 = the group runs on the whole grid with
                                              device barriers; k in 1..16 = the group runs in one
                                              thread-block cluster of k CTAs with cluster
                                              barriers (for narrow layers) */
    int32_t group_block[SPDZ_MAX_GROUPS];  /* per-group threads per CTA; 0 = plan value */
    uint32_t poll_ns;                      /* tagged: first sleep between polls of an operand
                                              that is not ready (ns, doubling up to 16x);
                                              0 = 128, at most 50000 */
    uint32_t barrier_slack;                /* tagged: a CTA starts the next layer once all but
                                              this many CTAs' arrivals are counted (operands
                                              still in flight validate by tag); 0 = a full
                                              barrier, at most the grid size */
    int32_t test_unwritten_tag;            /* testing, tagged mode only: 1 makes the first operand
                                              of every gate after the first layer wait for a tag
                                              that no store writes, so the bounded operand wait
                                              runs out (SPDZ_ERR_TIMEOUT); 0 in normal use */
    int32_t group_tagged[SPDZ_MAX_GROUPS]; /* fused, p = 2^61-1: 1 = the group runs the tagged
                                              kernel (as SPDZ_SCHED_TAGGED, over the group's layers,
                                              with barrier_slack and poll_ns); its first layer reads
                                              its operands from the wires the earlier groups
                                              finished, its later layers read the group's own
                                              outputs from the tagged copy.  group_cluster must be 0 */
} spdz_plan;

typedef struct {
    double device_ms;     /* device time of the run (CUDA events around it) */
    int32_t passed;       /* MAC-check verdict of the run */
    int32_t launches;     /* kernels the run executed (inside its graph, if captured) */
    int64_t n_gates;
    int64_t n_mul;
} spdz_stats;

/* Uploads and validates a circuit (every operand wire must come from an
 * earlier layer or the inputs; SPDZ_ERR_ARG otherwise).  The circuit is bound
 * to ctx's field and party count. */
int spdz_dag_create(spdz_ctx *ctx, const spdz_dag_desc *desc, spdz_dag **out);
int spdz_dag_destroy(spdz_dag *dag);

/* Evaluates the circuit on wires (a [n][>= n_inputs + n_gates] shared array
 * with the inputs filled in; gate outputs are written), consuming n_mul
 * triples, then runs the MAC check over everything the run opened.  Needs an
 * empty check epoch (SPDZ_ERR_STATE otherwise).  plan == NULL lets the
 * scheduler choose (learned cost model, else autotuned, else a fused
 * default).  With stats != NULL the call synchronises and fills it, and
 * returns SPDZ_ERR_MAC if the check failed; with stats == NULL the run is
 * only enqueued and spdz_check_result() reads the verdict later.
 * SPDZ_ERR_TIMEOUT: a device barrier wait hit its bound (results invalid). */
int spdz_run_dag(spdz_ctx *ctx, spdz_dag *dag, const spdz_plan *plan, const spdz_buf *wires,
                 spdz_stats *stats);
/* The same run from host buffers, for callers whose shares live in host
 * memory (p = 2^61-1 and p = 2^127-1, whose host and device element formats
 * agree; SPDZ_ERR_ARG for p = 2^32-5).  Enqueues, without waiting:
 *   - the run's n_mul triples, host arrays tri_host[0..5] = a, gamma(a), b,
 *     gamma(b), c, gamma(c), each [n][n_mul] (party rows of n_mul elements),
 *     copied into the registered pool at the slots the run consumes, on a
 *     copy stream of the context that waits only for the work enqueued before
 *     the pool was registered (so the next call's copy overlaps this run);
 *   - the input shares in_val_host / in_mac_host ([n][n_inputs] each) into
 *     wires, then the run (as spdz_run_dag with stats == NULL), on the
 *     context's stream;
 *   - wires [out_first, out_first + out_count) of every party (values and
 *     MACs) back to out_val_host / out_mac_host ([n][out_count] each).
 * Every host buffer must stay valid and unchanged until the stream has
 * passed this run (spdz_check_result synchronises); copies are asynchronous
 * only from and to page-locked host memory.  Errors as spdz_run_dag. */
int spdz_run_dag_host(spdz_ctx *ctx, spdz_dag *dag, const spdz_plan *plan, const spdz_buf *wires,
                      const void *in_val_host, const void *in_mac_host, const void *const *tri_host, int64_t out_first,
                      int64_t out_count, void *out_val_host, void *out_mac_host);
/* Verdict and sigma (host, [n] elements, may be NULL) of the last completed
 * check on the context; synchronises the stream. */
int spdz_check_result(spdz_ctx *ctx, int *passed, void *sigma_host);
/* Per-layer device times (microseconds, [depth]) of the last run that had
 * record_layer_times set. */
int spdz_dag_layer_times(const spdz_dag *dag, float *us_out);
/* Kernel timing of a circuit's runs (a measurement aid beside the run-time
 * figures of Sec. IV-B).  With on != 0 every later run of dag records CUDA
 * events on its stream right after its begin kernel and right after its last
 * circuit kernel (its check kernel included when the plan has one; a tagged
 * run checks inside its circuit kernel), also inside a captured graph: a
 * graph captured with the other setting is captured again at the next run.
 * spdz_dag_kernel_ms waits for the last such run and writes the time between
 * the two events (milliseconds) to *ms.  SPDZ_ERR_STATE when timing was never
 * enabled, SPDZ_ERR_CUDA when no timed run has completed. */
int spdz_dag_time_kernels(spdz_dag *dag, int32_t on);
int spdz_dag_kernel_ms(spdz_dag *dag, float *ms);
/* Layer-shape summary used by schedulers: for each layer l, counts[l*5 + c]
 * is the number of gates of class c (MUL, ADD, SUB, CMUL, CADD). */
int spdz_dag_layer_counts(const spdz_dag *dag, int32_t *counts_out);

/* ------------------------------------------------ allocation-free batch
 * No counterpart in the paper: an interface addition for callers that cannot
 * allocate device memory -- for example a host program whose own memory
 * manager has reserved the whole device, a plugin that is handed buffers but
 * no right to allocate, or a loop that cannot afford the device-wide
 * synchronisation cudaMalloc may cause.  Such callers cannot create a context
 * (which owns a small device workspace), so this call runs a Beaver batch
 * (same formulas and results as spdz_mul_batch) and the MAC check of its
 * opened values (same sigma as spdz_mac_check) without a context and without
 * allocating: it calls no cudaMalloc, cudaFree or allocating library routine.
 *
 * Arguments: n_parties (2..SPDZ_MAX_PARTIES), field, stream (cudaStream_t);
 * x, y: the N input pairs; a, b, c: the triples to consume, each view starting
 * at the first triple used (the caller tracks which triples are spent; a
 * triple must never be used twice); alpha_shares_dev: [n] alpha shares; z:
 * the N products (written); check_seed and epoch select the check's
 * coefficients exactly as a context's epoch `epoch` under spdz_set_check_seed
 * (opened eps_j at index 2j, delta_j at 2j+1); result_dev: [n + 1] elements,
 * written on the device: sigma_0 .. sigma_{n-1}, then 1 if the check passed and
 * 0 if it failed (the caller must then abort).  All device pointers are the
 * caller's; the call only enqueues work on `stream` and does not synchronise.
 *
 * Scratch: a fixed 4096-byte array compiled into the library (one per device
 * that loads it, held until the process exits), sized for the accumulators
 * of at most SPDZ_MAX_PARTIES parties; more parties are rejected with
 * SPDZ_ERR_ARG.  The first call on a device looks up the array's device
 * address (one cudaGetSymbolAddress, with that device current); make that
 * first call before any stream capture.  The address is kept until the
 * process exits, so do not call this entry point on a device after
 * cudaDeviceReset has torn down its context.  Every call shares the array and
 * clears it at its start: calls that overlap on the GPU (on different
 * streams, or from several host threads) race and give wrong results, so
 * order them on one stream.
 * Errors: SPDZ_ERR_ARG, SPDZ_ERR_ALIGN, SPDZ_ERR_CUDA (no message string: there
 * is no context). */
int spdz_mul_check_noalloc(int n_parties, int field, void *stream, const spdz_buf *x,
                           const spdz_buf *y, const spdz_buf *a, const spdz_buf *b,
                           const spdz_buf *c, const void *alpha_shares_dev, const spdz_buf *z,
                           int64_t N, uint64_t check_seed, uint64_t epoch, void *result_dev);

/* ------------------------------------------------------ learned cost model
 * The scheduler's cost model (the autotuning the paper leaves to future work,
 * Sec. V-D): a fully connected network n_in -> hidden x hidden_layers -> 1
 * with ReLU, FP32, trained on the device by the library's own forward,
 * backward (mean squared error) and Adam kernels.  Parameters are one flat
 * float array: per layer, W[out][in] row-major then b[out].  Initial weights
 * are He-uniform from the counter PRG under `seed`, biases zero.
 * X is [B][n_in] and targets/outputs [B], all float32 on the device. */
typedef struct spdz_mlp spdz_mlp;
int spdz_mlp_create(spdz_mlp **out, int32_t n_in, int32_t hidden, int32_t hidden_layers, uint64_t seed,
                    void *stream);
int spdz_mlp_destroy(spdz_mlp *m);
int spdz_mlp_num_params(const spdz_mlp *m, int64_t *count);
/* Copy the parameters out / in (host float arrays of spdz_mlp_num_params
 * entries); setting them also resets the Adam state.  Synchronise. */
int spdz_mlp_get_params(const spdz_mlp *m, float *host_out);
int spdz_mlp_set_params(spdz_mlp *m, const float *host_in);
int spdz_mlp_forward(spdz_mlp *m, const float *X_dev, int64_t B, float *Y_dev);
/* Mean squared error over the batch and its gradient (host outputs, either
 * may be NULL); synchronises. */
int spdz_mlp_loss_grad(spdz_mlp *m, const float *X_dev, const float *T_dev, int64_t B, float *loss_host,
                       float *grad_host);
/* Adam (beta1 0.9, beta2 0.999, eps 1e-8, step lr) for `epochs` passes over
 * consecutive mini-batches of `batch` rows; *loss_host (optional) receives the
 * final mean squared error over all B rows. */
int spdz_mlp_train(spdz_mlp *m, const float *X_dev, const float *T_dev, int64_t B, int32_t epochs,
                   int32_t batch, float lr, float *loss_host);
/* One Adam step (as in spdz_mlp_train, Kingma and Ba 2015, Algorithm 1) on
 * the caller's gradient grad_dev (device, spdz_mlp_num_params floats): the
 * step counter t advances by one, the moments m, v are updated and the
 * parameters move by lr * mhat / (sqrt(vhat) + 1e-8) with the bias
 * corrections 1 - 0.9^t and 1 - 0.999^t.  Enqueued on the model's stream. */
int spdz_mlp_adam_step(spdz_mlp *m, const float *grad_dev, float lr);

/* ---------------------------------------------------------- scheduling
 * Execution plans for circuit runs (the slice/batch-size autotuning and
 * profile-guided selection the paper leaves to future work, Sec. V-D).  A
 * plan never changes a result bit.  Every call below that runs the circuit
 * consumes triples from the context's pool (one run's worth per run) and needs
 * an empty check epoch, like spdz_run_dag.
 *
 * Candidate group configurations (index 0..count-1, spdz_sched_num_configs):
 * whole-grid groups with device barriers at several block sizes and CTAs per
 * SM, single-cluster groups (cluster barriers) for narrow layers, and (p =
 * 2^61-1) a tagged group (fence-free barriers over the tagged copy, a slack
 * of 1/12 of the CTAs).  The autotuner measures every configuration as one
 * group over the whole circuit; the learned planner mixes them per group. */
typedef struct {
    double default_ms;     /* measured makespan of the default fused plan */
    double autotuned_ms;   /* best measured makespan over the uniform configurations */
    double learned_ms;     /* measured makespan of the learned plan (-1: model not trained) */
    double predicted_ms;   /* the cost model's prediction for the learned plan (-1: none) */
    double switch_us;      /* measured cost of one extra layer group */
    int32_t chosen;        /* plan kept for plan == NULL runs: 0 default, 1 autotuned, 2 learned */
    int32_t learned_groups;
    int32_t samples;       /* training samples recorded so far */
    float train_loss;      /* final training loss (mean squared error of ln microseconds) */
    double tagged_ms;      /* measured makespan of the uniform tagged configuration (-1: not p61) */
    int32_t learned_is_autotuned; /* 1 when the learned plan is the autotuned uniform plan itself */
} spdz_sched_report;

int spdz_sched_num_configs(int32_t *count, int32_t *n_features);
/* The plan that runs the whole circuit as one group in configuration cfg. */
int spdz_sched_config_plan(const spdz_dag *dag, int32_t cfg, spdz_plan *out);
/* Runs the circuit under every configuration (1 + reps runs each) with
 * per-layer device timing and adds one sample per layer and configuration
 * (features -> ln of the median layer microseconds) to the context's training
 * set; the first call also measures the cost of one extra layer group. */
int spdz_sched_record(spdz_ctx *ctx, spdz_dag *dag, const spdz_buf *wires, int32_t reps);
/* The recorded samples (host arrays of count x n_features and count floats,
 * either may be NULL) and the measured group-switch cost. */
int spdz_sched_samples(spdz_ctx *ctx, float *X_host, float *Y_host, int64_t *count, double *switch_us);
/* Adds samples (for example recorded on a context of the other field) to the
 * context's training set: X_host [count][n_features], Y_host [count]. */
int spdz_sched_add_samples(spdz_ctx *ctx, const float *X_host, const float *Y_host, int64_t count);
/* Trains the context's cost model on the GPU (Adam, mini-batches of 128,
 * `epochs` passes, step lr) on every recorded sample; seed fixes the initial
 * weights and the sample order. */
int spdz_sched_train(spdz_ctx *ctx, int32_t epochs, float lr, uint64_t seed, float *loss_out);
/* Predicted microseconds of every layer ([depth]) under configuration cfg. */
int spdz_sched_predict(spdz_ctx *ctx, spdz_dag *dag, int32_t cfg, float *us_out);
/* The learned plan: group boundaries and per-group configurations that
 * minimise the predicted makespan (dynamic programming over the layers). */
int spdz_sched_learned_plan(spdz_ctx *ctx, spdz_dag *dag, spdz_plan *out, double *predicted_ms);
/* The autotuned plan: the fastest measured uniform configuration. */
int spdz_sched_autotune(spdz_ctx *ctx, spdz_dag *dag, const spdz_buf *wires, int32_t reps, spdz_plan *out,
                        double *best_ms);
/* Measures the default, autotuned and (if trained) learned plans, keeps the
 * fastest for this circuit's plan == NULL runs (the learned plan when it is
 * the autotuned plan itself), and reports them all. */
int spdz_sched_choose(spdz_ctx *ctx, spdz_dag *dag, const spdz_buf *wires, int32_t reps, spdz_plan *out,
                      spdz_sched_report *rep);

/* ------------------------------------------------------------- serving
 * A server for circuit requests (n parties; circuits over p = 2^61-1 or
 * p = 2^127-1, mixed freely; other fields are SPDZ_ERR_ARG), after the
 * paper's non-blocking scheduler over independently ready work (Sec. III-C)
 * applied across requests.  spdz_serve_start starts the server on a host
 * thread of its own; from then on callers submit requests at any time
 * (spdz_serve_submit returns at once with the request's id) and collect each
 * result when it is ready (spdz_serve_poll); spdz_serve_stop waits for every
 * submitted request to complete, then stops the thread.  Requests are
 * admitted first come, first served while the device-memory budget and
 * max_active slots allow: one arena of budget_bytes, allocated at creation,
 * holds every registered circuit's gate records and every admitted
 * request's wire shares, triples and (one-off circuits) gate records.  Each
 * admitted request's preprocessing is dealt on the device from its seed
 * (dealer kinds as spdz_deal_*: alpha, triples, and circuit inputs with
 * kind INPUT, sub 16, unless the caller passes the input shares) on an
 * offline stream, and its shares stay on the device until it completes.
 * Execution:
 *   SPDZ_SERVE_SEQUENTIAL: one request at a time, one launch per layer;
 *   SPDZ_SERVE_BATCHED: continuous batching -- each tick is one launch per
 *     field evaluating the next layer of every active request, and requests
 *     that arrive while others run join at the next tick;
 *   SPDZ_SERVE_HEURISTIC: as BATCHED, but a request whose widest layer has at
 *     most cluster_width gates runs all its layers in one cluster launch on a
 *     side stream, overlapping the ticks, and a request of at least 2^20
 *     gates runs all its layers in one fused launch with device barriers
 *     between layers (a cooperative launch on half the SMs' worth of CTAs)
 *     on a side stream;
 *   SPDZ_SERVE_LEARNED: as HEURISTIC, but the cluster or the grid launch is
 *     chosen when the cost model of model_ctx (trained with
 *     spdz_sched_train) predicts it to finish first, counting the launches of
 *     that kind already waiting.
 * Every request is its own MAC-check epoch (key of epoch 0 under
 * check_seed); its result does not depend on the mode or on the other
 * requests.  While the server runs, model_ctx belongs to the server thread:
 * the caller must not use it.  A CUDA failure ends the session: every request
 * not completed reports it, and later calls return it. */
enum spdz_serve_mode { SPDZ_SERVE_SEQUENTIAL = 0, SPDZ_SERVE_BATCHED = 1, SPDZ_SERVE_HEURISTIC = 2,
                       SPDZ_SERVE_LEARNED = 3 };

typedef struct spdz_server spdz_server;

typedef struct {
    const spdz_dag_desc *dag;   /* a one-off circuit (read during spdz_serve_submit; its gate
                                   records then live in the request's arena block), or NULL */
    int64_t circuit_id;         /* a circuit registered with spdz_serve_register, or -1 */
    int32_t field;              /* SPDZ_F61 or SPDZ_F127 (a registered circuit's own field) */
    uint64_t seed;              /* dealer seed of the request (alpha, triples, inputs) */
    double arrival_s;           /* spdz_serve_run: arrival time in seconds after the start
                                   (non-decreasing); spdz_serve_submit: 0 = now, or a past
                                   time after the start */
    const void *in_val_host;    /* optional: the input wires' value shares, host [n][n_inputs]
                                   elements, MACed under the alpha of `seed`; read when the
                                   request is admitted, so it must stay valid until the
                                   request completes.  NULL: dealt from the seed */
    const void *in_mac_host;    /* the input wires' MAC shares (required with in_val_host) */
    void *out_val_host;         /* optional: receives the request's wire value shares [n][W]
                                   (W = n_inputs + n_gates), written before it completes */
    void *out_mac_host;         /* optional: receives its wire MAC shares [n][W] */
} spdz_serve_request;

typedef struct {
    double latency_s;           /* arrival -> result available on the host */
    double online_s;            /* preprocessing dealt -> result */
    int32_t passed;             /* MAC-check verdict */
    int32_t mode;               /* 0 ticks, 1 cluster launch, 2 grid launch */
    int32_t status;             /* SPDZ_OK; SPDZ_ERR_MAC (check failed); SPDZ_ERR_OOM (can never
                                   fit the budget: refused); SPDZ_ERR_CUDA (session failed) */
    int32_t pad;
    uint64_t req_id;
} spdz_serve_result;

typedef struct {
    double wall_s, gates_per_s, p50_s, p99_s, mean_s;
    int64_t requests, gates, ticks, cluster_requests;
    double dealer_s;            /* device time spent dealing preprocessing (offline) */
    int64_t peak_bytes;         /* peak arena use of the session (registered circuits included) */
    int32_t max_active;
    /* host time of the serving thread by phase (tracing) */
    double host_admit_s, host_tick_s, host_complete_s, host_idle_s, host_ring_wait_s;
    /* device time of the ticks (events around each tick's launches), over
       device_ticks_timed ticks */
    double device_tick_s;
    int64_t device_ticks_timed;
    int64_t grid_requests;      /* requests run as one grid launch (mode 2) */
} spdz_serve_stats;

/* Creates a stopped server on the current device.  Errors: SPDZ_ERR_ARG,
 * SPDZ_ERR_OOM (the arena or the slot state cannot be allocated). */
int spdz_serve_create(spdz_server **out, int n_parties, uint64_t budget_bytes, int32_t max_active, int32_t mode,
                      spdz_ctx *model_ctx, uint64_t check_seed, int64_t cluster_width);
/* Registers a circuit of `field` (validated as spdz_dag_create; read during
 * the call) for any number of requests: its gate records are uploaded into
 * the arena, counted against the budget, and stay until unregistered.  Only
 * while stopped (SPDZ_ERR_STATE).  Errors: SPDZ_ERR_ARG, SPDZ_ERR_OOM (no room
 * left in the budget). */
int spdz_serve_register(spdz_server *s, const spdz_dag_desc *dag, int32_t field, int64_t *circuit_id);
int spdz_serve_unregister(spdz_server *s, int64_t circuit_id);
/* Changes the execution mode (only while stopped). */
int spdz_serve_set_mode(spdz_server *s, int32_t mode, spdz_ctx *model_ctx, int64_t cluster_width);
/* Starts the serving thread (SPDZ_ERR_STATE when already running); the
 * statistics of spdz_serve_stop cover the requests completed from here. */
int spdz_serve_start(spdz_server *s);
/* Submits one request (thread-safe; returns without waiting).  Exactly one of
 * r->dag and r->circuit_id >= 0 names the circuit.  The host buffers the
 * request points to must stay valid until spdz_serve_poll reports it done.
 * Errors: SPDZ_ERR_ARG (bad circuit, field or buffers), SPDZ_ERR_STATE (not
 * running). */
int spdz_serve_submit(spdz_server *s, const spdz_serve_request *r, uint64_t *req_id);
/* *done = 1 and *result filled once the request has completed (its outputs
 * are then in its host buffers); a result is handed out once.  *done = 0
 * while it is pending.  SPDZ_ERR_ARG for an unknown or collected id. */
int spdz_serve_poll(spdz_server *s, uint64_t req_id, int32_t *done, spdz_serve_result *result);
/* Waits for every submitted request to complete, stops the thread and fills
 * stats (may be NULL) over the session's completed requests; results not yet
 * collected stay available to spdz_serve_poll. */
int spdz_serve_stop(spdz_server *s, spdz_serve_stats *stats);
/* Trace driver over the calls above: starts the server, submits each request
 * at its arrival_s (seconds after the start) from the calling thread, stops,
 * and collects results [count] (may be NULL).  Returns the first failing
 * request status (for example SPDZ_ERR_OOM for a request that can never fit). */
int spdz_serve_run(spdz_server *s, const spdz_serve_request *reqs, int64_t count, spdz_serve_result *results,
                   spdz_serve_stats *stats);
/* Stops the server if it runs, then frees everything it holds. */
int spdz_serve_destroy(spdz_server *s);

/* ------------------------------------------------------- matrix products
 * Secret-shared matrix products with Beaver matrix triples (Sec. III-D.3:
 * one triple (A, B, C = A*B) per product).  Matrices are row-major inside
 * each party row of a spdz_buf (element (r, c) of party i at ptr + i*stride +
 * r*cols + c).  p = 2^61 - 1 only. */
enum spdz_matmul_path {
    SPDZ_MATMUL_CUDA_CORE = 0,   /* 64-bit modular multiply-accumulate on the CUDA cores */
    SPDZ_MATMUL_TENSOR = 1       /* exact small-digit products on the tensor cores */
};
/* Dealer for one matrix triple: A (m x k) and B (k x n) uniform (kinds
 * MTRIPLE_A/B, element index = row-major position, stream sub `sub`),
 * C = A*B (kind MTRIPLE_C), each shared with MACs under alpha_shares_dev. */
int spdz_deal_matrix_triple(spdz_ctx *ctx, uint64_t seed, uint64_t sub, int64_t m, int64_t k, int64_t n,
                            const void *alpha_shares_dev, const spdz_buf *A, const spdz_buf *B, const spdz_buf *C);
/* Registers one matrix triple (referenced, not copied) for the next
 * spdz_matmul of the same shape; a triple is consumed by one product. */
int spdz_load_matrix_preproc(spdz_ctx *ctx, const spdz_buf *A, const spdz_buf *B, const spdz_buf *C, int64_t m,
                             int64_t k, int64_t n);
/* Z = X * Y on shares: opens E = X - A and F = Y - B (their MAC shares join
 * the current check epoch, E row-major first, then F), then
 *   Z_i = C_i + E*B_i + A_i*F + [i == 0] E*F,
 *   gamma(Z)_i = gamma(C)_i + E*gamma(B)_i + gamma(A)_i*F + alpha_i E*F.
 * E_out_dev / F_out_dev (device, m*k and k*n elements, may be NULL) receive
 * the opened matrices.  SPDZ_ERR_TRIPLES without a registered triple of this
 * shape. */
int spdz_matmul(spdz_ctx *ctx, const spdz_buf *X, const spdz_buf *Y, const spdz_buf *Z, int64_t m, int64_t k,
                int64_t n, int path, void *E_out_dev, void *F_out_dev);

/* ------------------------------------------------------ inputs, outputs
 * The steps on either side of the online core (Sec. I: parties secret-share
 * their private inputs and combine shares of the result only to reveal the
 * output; Sec. II-A.2: revealed values are accepted after the MAC check;
 * Sec. IV: every input is secret-shared before the computation). */
/* Dealer for input masks of party `owner`: r uniform (kind INPUT_MASK, stream
 * sub = owner, element index j0 + j), shared with MACs into masks, and the
 * clear r (which only the owner holds) into r_clear_dev ([count] elements,
 * device). */
int spdz_deal_input_masks(spdz_ctx *ctx, uint64_t seed, int32_t owner, uint64_t j0, int64_t count,
                          const void *alpha_shares_dev, const spdz_buf *masks, void *r_clear_dev);
/* Secret-shares the owner's private inputs x_dev ([N] canonical elements,
 * device) with its masks: the owner publishes eps = x - r (written to
 * eps_out_dev when not NULL) and out = [r] + eps, i.e. party 0's value share
 * gets + eps and every party's MAC share + alpha_i * eps.  Each mask must be
 * used once (the caller tracks them).  Needs the alpha shares loaded. */
int spdz_input(spdz_ctx *ctx, const void *x_dev, const void *r_clear_dev, const spdz_buf *masks, const spdz_buf *out,
               int64_t N, void *eps_out_dev);
/* Reveals N shared values: opens them into out_dev (device, [N] elements;
 * they join the check epoch), then runs the MAC check over the epoch
 * (spdz_mac_check).  On failure *passed = 0, out_dev is zeroed and the call
 * returns SPDZ_ERR_MAC: nothing is released.  sigma_host as spdz_mac_check. */
int spdz_reveal(spdz_ctx *ctx, const spdz_buf *x, void *out_dev, int64_t N, int *passed, void *sigma_host);

/* ---------------------------------------------------------- linear layer
 * The LinearLayer operator y = W x + b (Sec. III-D.3 "Data slicing" and
 * "MPC-specific optimization"; the workload of the paper's evaluation,
 * Sec. IV) on a secret-shared dout x din matrix W (row-major in each party
 * row), din vector x and dout vector b.  W is cut into tiles of tile_rows
 * consecutive rows (the last tile may be shorter; tile_rows above dout means
 * one tile), T = ceil(dout / tile_rows).  Tile t consumes one matrix-vector
 * triple: A_t = its rows of a dout x din matrix A, B_t (din values) and
 * C_t = A_t B_t (its tile_rows values).  The tile opens E_t = x - B_t and
 * D_t = W_t - A_t and every party computes
 *   z_i = C_i + D_t B_{t,i} + A_{t,i} E_t + [i == 0] D_t E_t,
 *   gamma(z)_i = gamma(C)_i + D_t gamma(B)_{t,i} + gamma(A)_{t,i} E_t + alpha_i D_t E_t,
 * then y_i = z_i + b_i and gamma(y)_i = gamma(z)_i + gamma(b)_i.  The opened
 * values join the current check epoch in this order: per tile, E_t (din
 * values), then D_t row by row.  p = 2^61 - 1 and p = 2^32 - 5 (SPDZ_ERR_ARG
 * otherwise).
 * Shapes of the triple buffers: A [n][dout*din], B [n][T*din] (B_t at
 * t*din), C [n][dout]. */
/* Dealer for the layer's triples: A and B uniform (kinds MTRIPLE_A/B,
 * element index = position in A, resp. t*din + k), C_t = A_t B_t (kind
 * MTRIPLE_C, index = row), each shared with MACs under alpha_shares_dev.
 * Uses a device workspace of (dout*din + T*din + dout) elements, kept by the
 * context. */
int spdz_deal_matvec_triples(spdz_ctx *ctx, uint64_t seed, uint64_t sub, int64_t dout, int64_t din, int64_t tile_rows,
                             const void *alpha_shares_dev, const spdz_buf *A, const spdz_buf *B, const spdz_buf *C);
/* Registers the triples (referenced, not copied) for the next
 * spdz_linear_layer of the same shape and tiling; one layer consumes them. */
int spdz_load_matvec_preproc(spdz_ctx *ctx, const spdz_buf *A, const spdz_buf *B, const spdz_buf *C, int64_t dout,
                             int64_t din, int64_t tile_rows);
/* y = W x + b as above.  D_out_dev (dout*din elements) and E_out_dev (T*din
 * elements), device, may be NULL: they receive the opened D (row-major) and
 * E (tile by tile).  SPDZ_ERR_TRIPLES without registered triples of this
 * shape and tiling. */
int spdz_linear_layer(spdz_ctx *ctx, const spdz_buf *W, const spdz_buf *x, const spdz_buf *b, const spdz_buf *y,
                      int64_t dout, int64_t din, int64_t tile_rows, void *D_out_dev, void *E_out_dev);

/* ------------------------------------------------------ party per GPU
 * One party of the online phase whose shares live on its own GPU (one
 * process and one GPU per party: the paper runs its parties as separate
 * processes, Sec. IV-A, and names a GPU per party as future work, Sec. V-B).
 * Only the party's own rows are touched; the exchange between parties (the
 * open: every party's eps_i, delta_i rows; the check: every sigma_i) is the
 * caller's, for example an all-gather over NCCL.  A Beaver batch is
 *   spdz_party_mask -> exchange -> spdz_party_open_sum -> spdz_party_combine
 * and the batched MAC check of an epoch is spdz_party_sigma on every party,
 * an exchange of the sigmas, and "pass iff they sum to zero mod p".  The
 * opened values, their check coefficients and the formulas are those of
 * spdz_mul_batch / spdz_mac_check (eps_j at epoch index 2j, delta_j at
 * 2j+1, coefficient key of epoch e under the check seed), so the parties
 * together compute exactly what one context computes for all of them.
 * Single-party buffers: spdz_buf with the party's value and MAC rows (stride
 * unused).  Every call enqueues on the party's stream; spdz_party_sigma
 * synchronises it.  Errors: SPDZ_ERR_ARG, SPDZ_ERR_ALIGN (an element
 * pointer not aligned to its element size), SPDZ_ERR_STATE, SPDZ_ERR_OOM,
 * SPDZ_ERR_CUDA. */
typedef struct spdz_party spdz_party;
int spdz_party_create(spdz_party **out, int party, int n_parties, int field, void *stream);
int spdz_party_destroy(spdz_party *p);
/* This party's MAC-key share alpha_i (device, one element); resets the
 * epoch's sums. */
int spdz_party_load_alpha(spdz_party *p, const void *alpha_share_dev);
/* Seed of the check coefficients; epoch 0 (SPDZ_ERR_STATE with values opened). */
int spdz_party_set_check_seed(spdz_party *p, uint64_t seed);
/* eps_i = x_i - a_i and delta_i = y_i - b_i (value rows, N elements each) into
 * eps_dev, dlt_dev: this party's contribution to the open. */
int spdz_party_mask(spdz_party *p, const spdz_buf *x, const spdz_buf *y, const spdz_buf *a, const spdz_buf *b,
                    void *eps_dev, void *dlt_dev, int64_t N);
/* out[j] = sum_k rows[k*N + j] over the n parties' gathered rows (device,
 * [n][N] contiguous): the opened public values. */
int spdz_party_open_sum(spdz_party *p, const void *rows_dev, int64_t N, void *out_dev);
/* With the public eps, delta ([N] each, device): z_i and gamma(z)_i as in
 * spdz_mul_batch for this party (party 0 adds eps delta to its value), and
 * the check sums A += r eps + r' delta, S_i += r (gamma(x)_i - gamma(a)_i)
 * + r' (gamma(y)_i - gamma(b)_i) for the 2N values opened. */
int spdz_party_combine(spdz_party *p, const void *eps_dev, const void *dlt_dev, const spdz_buf *x, const spdz_buf *y,
                       const spdz_buf *a, const spdz_buf *b, const spdz_buf *c, const spdz_buf *z, int64_t N);
/* sigma_i = S_i - alpha_i A over the epoch (host, one element; two 64-bit
 * words for p127), *opened_out (may be NULL) = values opened in it; then
 * the next epoch starts.  Synchronises the party's stream. */
int spdz_party_sigma(spdz_party *p, void *sigma_host, int64_t *opened_out);

/* ------------------------------------------------------------ measurement
 * Integer issue-rate microbenchmark (no counterpart in the paper; the
 * compute-side denominator of the roofline of kernels bound by integer
 * arithmetic, such as the p = 2^127-1 products): every thread of a grid of
 * 8 CTAs x 256 threads per SM runs eight independent chains of one
 * instruction kind for `iters` x 4 rounds:
 *   kind 0: 32-bit multiply-add, low half (mad.lo.u32);
 *   kind 1: 32 x 32 + 64 -> 64 multiply-add (mad.wide.u32);
 *   kind 2: high half of a 32 x 32 product then an add (mul.hi.u32, add.u32);
 *   kind 3: integer add then xor (add.u32, xor.b32).
 * *ops_per_s receives thread-level instructions per second (both
 * instructions of a kind-2 or kind-3 pair counted).  scratch_dev: device
 * buffer of at least 8 x 256 x SMs uint32 (written).  Synchronises the
 * stream.  Errors: SPDZ_ERR_ARG, SPDZ_ERR_CUDA. */
int spdz_int_peak(int kind, int64_t iters, void *stream, void *scratch_dev, double *ops_per_s);

#ifdef __cplusplus
}
#endif

#endif /* SPDZ_H */
