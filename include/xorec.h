/*
 * xorec: XOR-based Reed-Solomon erasure coding on one GB300 GPU.
 *
 * C ABI of libxorec.so.  Plain pointers and sizes only.
 *
 * Method (paper: Uezato, "Accelerating XOR-based Erasure Coding using
 * Program Optimization Techniques", SC'21):
 *   - RS(k,m) encodes k data blocks into m parity blocks with the systematic
 *     generator [I ; P] over GF(2^8), polynomial 0x11d (Sec. 1, Sec. 7.1).
 *   - The m x k parity matrix is expanded into an (8m) x (8k) bitmatrix over
 *     GF(2) (Sec. 1, properties (i)-(ii)); every output strip is the XOR of
 *     the input strips its bitmatrix row selects.
 *   - The bitmatrix becomes a straight-line program (Sec. 4.1) that is
 *     compressed by XorRePair (Sec. 4.4), fused (Sec. 5.2) and scheduled by
 *     a pebble game (Sec. 6.6) before it runs on the GPU.
 *
 * Data layout.  A block of B bytes (B % 128 == 0) is 8 strips of B/8 bytes;
 * strip t is bytes [t*B/8, (t+1)*B/8).  Bit t of field element e is bit
 * (e % 8) of byte e/8 of strip t (Sec. 6.1 "8 x n arrays of N/(8n) bytes").
 * Block pointers must be 16-byte aligned.
 *
 * Ownership.  The caller owns every data buffer; a plan owns its host
 * programs and device state and must outlive the GPU work queued with it.
 * Calls that take a stream are asynchronous with respect to the host;
 * argument errors are returned synchronously.  Errors found by kernels
 * (a bounded wait that timed out) are reported by ec_device_status(); a
 * batch also records them in its own word (ec_batch_status) and a server
 * fails the requests of the affected batch (ec_server_poll_ex).
 * ec_last_error() returns a thread-local message for the last failure.
 *
 * Threads.  Encode, decode, batch and serving calls may run from several
 * host threads at once, also on one plan (decoders and compiled kernels are
 * built once, under the plan's lock); ec_plan_autotune, ec_plan_set_launch
 * and ec_plan_destroy must not overlap other calls on the same plan.
 */
#ifndef XOREC_H
#define XOREC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  EC_OK = 0,
  EC_EINVAL = -1,      /* bad argument (sizes, alignment, ids)                */
  EC_ENOMEM = -2,      /* host or device allocation failed                    */
  EC_ESINGULAR = -3,   /* survivor submatrix not invertible (non-MDS matrix)  */
  EC_ETOOMANY = -4,    /* more erasures than parity blocks                    */
  EC_ECUDA = -5,       /* CUDA runtime / driver error                         */
  EC_ETIMEOUT = -6,    /* a device-side bounded wait gave up                  */
  EC_EBUSY = -7,       /* admission refused (serving)                         */
  EC_ENOTSUP = -8      /* feature unavailable (e.g. no run-time compiler)     */
} ec_status;

typedef struct ec_plan ec_plan;

/* Coding-matrix choice for ec_plan_create_ex. */
enum {
  EC_MATRIX_CAUCHY = 0, /* P[i][j] = 1 / ((k+i) XOR j): MDS for k+m <= 256   */
  EC_MATRIX_POWER = 1,  /* P[r][j] = 2^(r*j): the matrix whose XOR counts the
                           paper prints for RS(10,4) (Sec. 7.1, Sec. 7.5);
                           not MDS in general                                 */
  EC_MATRIX_USER = 2,   /* caller-supplied m x k parity rows, used as given   */
  EC_MATRIX_CAUCHY_MIN = 3 /* the Cauchy rows and columns scaled by nonzero
                           constants to few bitmatrix ones (the XOR count
                           depends on the matrix, Sec. 7.6): each column
                           divided by its row-0 entry (row 0 = all ones),
                           then each later row divided by the entry of that
                           row leaving the fewest ones (ties: smallest
                           entry).  MDS like the Cauchy matrix; its parity
                           bytes differ from EC_MATRIX_CAUCHY's          */
};

/* Optimiser level (which passes run before fusion and scheduling). */
enum {
  EC_OPT_RAW = 0,       /* one fused statement per bitmatrix row              */
  EC_OPT_REPAIR = 1,    /* RePair (Sec. 4.3)                                  */
  EC_OPT_XORREPAIR = 2, /* XorRePair (Sec. 4.4), the default                  */
  EC_OPT_TRIPLE = 3     /* RePair's greedy compression with triples of terms
                           (one three-input XOR instruction each) in place of
                           pairs; codes too wide to enumerate triples use
                           XorRePair                                          */
};

/* Pebble-game scheduler (Sec. 6.6). */
enum { EC_SCHED_DFS = 0, EC_SCHED_GREEDY = 1 };

/* Executor tier.  Without a compiled kernel (none yet, no run-time
 * compiler, or a program too large for one) EC_EXEC_AUTO runs the dense
 * bitmatrix executor: output strip r = XOR of the input strips c whose bit
 * (r, c) of the program's bitmatrix is set (Sec. 1, property (ii)), built
 * into the library. */
enum {
  EC_EXEC_AUTO = 0,     /* compiled straight-line kernel, else dense          */
  EC_EXEC_INTERP = 1,   /* instruction-stream interpreter of the SLP          */
  EC_EXEC_COMPILED = 2, /* compiled straight-line kernel (NVRTC)              */
  EC_EXEC_DENSE = 3     /* dense bitmatrix executor                           */
};

typedef struct {
  int opt_level;        /* EC_OPT_*                                           */
  int sched;            /* EC_SCHED_*                                         */
  int greedy_cap;       /* cache capacity of the greedy scheduler             */
  int executor;         /* EC_EXEC_*                                          */
  int max_temps;        /* (Xor)RePair temporaries budget: -1 = unlimited
                           (the paper's full run), -2 = automatic, >= 0 =
                           explicit (0 = one fused statement per row).  The
                           most frequent pairs are factored first, so a
                           budget keeps the most valuable temporaries while
                           bounding the registers the program needs          */
  int reg_budget;       /* registers per thread the automatic budget aims at
                           (all input words preloaded); 0 = 128, else in
                           [32, 255].  Above 128 it also raises the compiled
                           kernels' register cap (fewer CTAs per SM), as
                           ec_plan_set_launch does                          */
  int stream_window;    /* codes with more than 96 input strips (12 data
                           blocks) and automatic temporaries: the input words
                           do not fit the registers, so the program is
                           two-level (Sec. 8's multilevel pebble game): rows
                           in groups of partial sums that fit reg_budget,
                           inputs in windows of this many strips, each input
                           word read from the shared-memory tile once per
                           group, two inputs per three-input XOR.  0 =
                           automatic (32), -1 = off (one fused statement per
                           row, operands read from shared memory at every
                           use), > 0 = explicit                            */
  int stream_temps;     /* two-level programs: XorRePair temporals per window
                           (Sec. 4.4 on each window's part of the rows, then
                           fusion); 0 = automatic (the planner tries 0, 8,
                           16 and 32 and keeps the cheapest that fits the
                           registers), -1 = none, > 0 = explicit            */
} ec_plan_opts;

/* Create a plan for RS(k,m).  matrix: m*k row-major parity rows, or NULL for
 * the Cauchy default.  1 <= k, 1 <= m, k + m <= 256.  Builds and optimises
 * the encoding program on the host (Sec. 4-6).  *out receives the plan. */
ec_status ec_plan_create(int k, int m, const uint8_t *matrix, ec_plan **out);

/* Same with an explicit matrix kind (EC_MATRIX_*; matrix is read only for
 * EC_MATRIX_USER) and options (NULL = defaults). */
ec_status ec_plan_create_ex(int k, int m, int matrix_kind, const uint8_t *matrix,
                            const ec_plan_opts *opts, ec_plan **out);

/* Free the plan, its programs and its device state.  NULL is ignored. */
void ec_plan_destroy(ec_plan *plan);

/* Copy the m*k parity rows of the plan into out (host memory). */
ec_status ec_plan_matrix(const ec_plan *plan, uint8_t *out);

/* Statistics of one program of the plan. */
typedef struct {
  long xors, mem;       /* #XOR (sum of arity-1) and #_M (Sec. 4.1, 5.1)      */
  int nvar, stmts;      /* variables and statements                           */
} ec_slp_stats;

typedef struct {
  int n_in, n_out;      /* input / output strips                              */
  int slots;            /* pebbles (slots) of the program's stream            */
  int stmts;            /* statements of the lowered program                  */
  int code_words;       /* 16-bit words of the program's instruction stream   */
  int sched_nvar;       /* pebbles of the paper's game (goals hold)           */
  ec_slp_stats raw;     /* unoptimised binary-chain program (Sec. 7.5)        */
  ec_slp_stats compressed;  /* after (Xor)RePair                              */
  ec_slp_stats fused;   /* after XOR fusion                                   */
  int compiled;         /* 1 if a compiled straight-line kernel exists        */
  int regs;             /* registers per thread of the compiled kernel        */
  int temps;            /* temporaries kept by (Xor)RePair                    */
  int max_live;         /* values live at once (inputs preloaded; two-level
                           programs: inputs live within their group)         */
  int threads;          /* threads per CTA of the compiled tier (strip tile =
                           4 x threads bytes): the plan's launch shape        */
  int lop3;             /* three-input XOR instructions of the fused program:
                           sum over statements of ceil((arity - 1) / 2)       */
  int loads;            /* input words a thread reads from the shared-memory
                           tile per tile: n_in when preloaded, once per group
                           for two-level programs, at every use otherwise     */
  int window;           /* input window of a two-level program, else 0       */
  int window_temps;     /* XorRePair temporals per window (two-level)        */
} ec_program_info;

/* Program of the encoder (erasures == NULL) or of the decoder for the given
 * erasure set (built and cached on first use). */
ec_status ec_plan_info(ec_plan *plan, const int *erasures, int n_erasures,
                       ec_program_info *out);

/* CUDA C++ source of the compiled tier's kernel for the encoder (erasures ==
 * NULL) or a decoder, as the plan compiles it at its launch shape (NVRTC,
 * sm_103a): the tile pipeline, the program's straight-line statements and
 * the kernel entry.  Copies at most len - 1 characters and a terminating NUL
 * into buf (NULL: none); *need receives the full length including the NUL.
 * Host only; for inspection and for checking the compile without a GPU. */
ec_status ec_plan_kernel_source(ec_plan *plan, const int *erasures, int n_erasures, char *buf,
                                size_t len, size_t *need);

/* CUDA C++ source of the multi-program module that batched launches compile
 * for the decoders of the given erasure sets (layout of ec_decode_prepare;
 * n_sets == 0: the encoder alone), at the plan's module launch shape: the
 * tile pipeline with its work queue, every program's straight-line
 * statements and the kernel entry.  The programs must share their input
 * count.  Copies at most len - 1 characters and a NUL into buf (NULL: none);
 * *need receives the full length including the NUL.  Host only; for
 * inspection and for checking the compile without a GPU. */
ec_status ec_plan_module_source(ec_plan *plan, const int *sets, const int *counts, int n_sets,
                                char *buf, size_t len, size_t *need);

/* Copy the instruction stream of the encoder's program (erasures == NULL)
 * or of a decoder's into buf (len 16-bit words); *need receives the length.
 * This is the optimised, scheduled program that the compiled tier runs, in
 * stream form.  Stream format, statement by statement: n_args; n_outs |
 * has_slot << 15; [slot]; output strip ids; operand ids (< n_in: input
 * strip, else slot + n_in).  The interpreter tier runs the same program,
 * except for codes of up to 96 input strips, where it runs the unoptimised
 * fused program (one statement per output strip, no slots): its tile of
 * inputs and slots lives in shared memory, and without slots twice as many
 * warps fit an SM.  For inspection and host-side checks. */
ec_status ec_plan_program(ec_plan *plan, const int *erasures, int n_erasures, uint16_t *buf,
                          size_t len, size_t *need);

/* Copy the dense bitmatrix executor's control words of the encoder's
 * program (erasures == NULL) or of a decoder's into buf (len 32-bit words);
 * *need receives their number, 2 * G * n_in with G = ceil(n_out / 32) groups
 * of output strips.  They encode the program's bitmatrix (Sec. 1, property
 * (ii): output strip r reads input strip c where bit (r, c) is set) twice:
 * first G * n_in column masks (word g * n_in + c, bit i: bit (32 g + i, c)),
 * then G * n_in row words (word g * n_in + 8 w + j, bit 8 q + i: bit
 * (32 g + 4 j + q, 8 w + i)).  For inspection and host-side checks. */
ec_status ec_plan_dense_words(ec_plan *plan, const int *erasures, int n_erasures, uint32_t *buf,
                              size_t len, size_t *need);

/* Encode one stripe: parity_i = sum_j P[i][j] data_j (Sec. 1).
 * data[k], parity[m]: device pointers to blocks of block_bytes bytes
 * (block_bytes % 128 == 0, 16-byte aligned).  Enqueued on `stream`
 * (a cudaStream_t, NULL = legacy default stream). */
ec_status ec_encode(ec_plan *plan, const uint8_t *const *data, uint8_t *const *parity,
                    size_t block_bytes, void *stream);

/* Limits of ec_encode_noalloc. */
#define EC_NOALLOC_MAX_BLOCKS 256        /* k + m                            */
#define EC_NOALLOC_MAX_CODE_WORDS 32768  /* 16-bit words of the program as the
                                            interpreter reads it on the device
                                            (its stream in 16-byte chunks)   */

/* Encode one stripe like ec_encode, without allocating any memory.  The
 * paper has no counterpart: this is for callers that are not allowed to
 * allocate device memory when they encode (code running inside another
 * runtime's allocator, or under a fixed device-memory budget planned in
 * advance).  Its scratch (status word, block table and instruction stream,
 * about 66 KiB) lives in one static device array that every GPU loading the
 * library keeps until the process exits.  All calls share that array and
 * each call overwrites it, so calls whose GPU work overlaps race.  The
 * first call on each device performs that device's set-up (looks up the
 * array's address, clears its status word) and should come before any
 * stream capture.  Always uses the interpreter executor.  A bounded wait
 * of its kernel that gives up is recorded in the array's status word, which
 * ec_device_status reads beside the device's own.  Fails with
 * EC_EINVAL when k + m > EC_NOALLOC_MAX_BLOCKS or the encoding program is
 * longer than EC_NOALLOC_MAX_CODE_WORDS.  Same arguments as ec_encode. */
ec_status ec_encode_noalloc(ec_plan *plan, const uint8_t *const *data, uint8_t *const *parity,
                            size_t block_bytes, void *stream);

/* Encode n_stripes stripes in one launch.  Block j of stripe s is at
 * data + s*data_stripe_stride + j*data_block_stride; parity block i of stripe
 * s at parity + s*par_stripe_stride + i*par_block_stride (bytes, device
 * memory, multiples of 16). */
ec_status ec_encode_strided(ec_plan *plan, const uint8_t *data, size_t data_stripe_stride,
                            size_t data_block_stride, uint8_t *parity,
                            size_t par_stripe_stride, size_t par_block_stride,
                            int n_stripes, size_t block_bytes, void *stream);

/* Encode n_stripes stripes that live in HOST memory (same strided layout as
 * ec_encode_strided, host addresses).  Chunks of chunk_stripes stripes (0 =
 * 16) are copied to device staging owned by the plan, encoded and their
 * parity copied back, on three internal streams so that both copy
 * directions and the kernels overlap.  Pinned host memory gives full link
 * speed; pageable memory works but copies synchronously.  Asynchronous with
 * respect to the host: the work is ordered after `stream`'s prior work and
 * `stream` waits for all of it; keep the buffers alive until then.  Calls
 * on one plan from several host threads are enqueued one at a time (they
 * share the plan's staging and streams). */
ec_status ec_encode_host_strided(ec_plan *plan, const uint8_t *data, size_t data_stripe_stride,
                                 size_t data_block_stride, uint8_t *parity,
                                 size_t par_stripe_stride, size_t par_block_stride,
                                 int n_stripes, size_t block_bytes, int chunk_stripes,
                                 void *stream);

/* Decode one stripe (Sec. 1): recover the blocks listed in erasures (ids in
 * [0, k+m), unique, any order, 1 <= n_erasures <= m) from the first k
 * surviving blocks in ascending id order.  blocks[k+m] is indexed by block
 * id (data blocks 0..k-1, parity blocks k..k+m-1); erased entries are
 * ignored and may be NULL.  out[i] receives block erasures[i]; erased parity
 * is re-encoded from the recovered data in the same program.  The decode
 * matrix G[E] * G[S]^{-1} is inverted on the host and its program built and
 * cached on first use of each erasure set. */
ec_status ec_decode(ec_plan *plan, const int *erasures, int n_erasures,
                    const uint8_t *const *blocks, uint8_t *const *out,
                    size_t block_bytes, void *stream);

/* Build (in parallel host threads) and cache the decode programs of
 * n_sets erasure sets.  sets holds the ids of all sets back to back;
 * counts[i] is the size of set i. */
ec_status ec_decode_prepare(ec_plan *plan, const int *sets, const int *counts, int n_sets,
                            int n_threads);

/* Compile, in parallel host threads, the straight-line kernels of the
 * encoder (n_sets == 0) or of the decoders of the given erasure sets (same
 * layout as ec_decode_prepare), so that later calls do not compile. */
ec_status ec_plan_compile(ec_plan *plan, const int *sets, const int *counts, int n_sets,
                          int n_threads);

/* Autotuner: times the encoder under candidate launch shapes (threads per
 * CTA, i.e. tile bytes per strip) and register budgets (which bound the
 * XorRePair temporaries) on n_stripes scratch stripes of block_bytes,
 * checks that every candidate writes identical parity, and installs the
 * fastest program in the plan; decoders built afterwards use the same
 * budget and shape.  Allocates scratch device memory for the duration of
 * the call and synchronises `stream`.  Must not run concurrently with other
 * calls on the same plan. */
typedef struct {
  int threads;           /* threads per CTA of the compiled tier            */
  int reg_budget;        /* register budget of the temporaries              */
  int min_ctas_per_sm;   /* occupancy the kernel was compiled for           */
  int candidates;        /* candidates timed                                */
  double ms;             /* best time per launch                            */
  double gbps_in;        /* best input throughput, GB/s                     */
} ec_tune_result;

ec_status ec_plan_autotune(ec_plan *plan, size_t block_bytes, int n_stripes, void *stream,
                           ec_tune_result *out);

/* Set the launch shape without timing: `threads` per CTA of the compiled
 * tier (a multiple of 32 in [32, 1024]; the strip tile is 4 x threads bytes)
 * and the register budget of the XorRePair temporaries ([32, 255]).  The
 * encoder is rebuilt with that budget; decoders and batch modules built
 * afterwards use the same budget and shape (the paper's cache-capacity
 * parameter, Sec. 6.2, retargeted to registers).  Host-only; EC_EINVAL for
 * values out of range.  Must not run concurrently with other calls on the
 * same plan. */
ec_status ec_plan_set_launch(ec_plan *plan, int threads, int reg_budget);

/* Select the executor tier (EC_EXEC_*).  EC_EXEC_COMPILED fails with
 * EC_ENOTSUP when no run-time compiler is present. */
ec_status ec_plan_set_executor(ec_plan *plan, int executor);

/* ------------------------------------------------------------------ batches
 * Many stripes with mixed codes, block sizes and encode/decode jobs run in a
 * few persistent launches.  The plans referenced by a batch must outlive
 * it; the job arrays only need to live until ec_batch_create returns. */
enum { EC_OP_ENCODE = 0, EC_OP_DECODE = 1 };

typedef struct {
  ec_plan *plan;
  int op;                          /* EC_OP_ENCODE or EC_OP_DECODE                */
  const int *erasures;             /* decode: erased block ids (caller order)     */
  int n_erasures;                  /* decode: 1 .. m                              */
  const uint8_t *const *blocks;    /* encode: k data blocks; decode: k+m blocks
                                      indexed by id (erased entries ignored)     */
  uint8_t *const *out;             /* encode: m parity blocks; decode:
                                      n_erasures blocks in the caller's order    */
  size_t block_bytes;              /* multiple of 128                             */
} ec_job;

typedef struct ec_batch ec_batch;

typedef struct {
  long long stripes, items;        /* jobs and 512-byte work items               */
  long long bytes_in, bytes_out;   /* block bytes read and written per run       */
  int programs;                    /* distinct programs                          */
  int compiled_programs;           /* of which run by compiled modules           */
  int launches;                    /* kernel launches per ec_batch_run           */
  int modules_built;               /* modules compiled by ec_batch_create        */
  double prepare_ms;               /* host time of ec_batch_create               */
} ec_batch_info;

/* Build the programs the jobs need (decode programs in parallel host
 * threads), compile those without a compiled form into multi-program
 * modules owned by their plan (executor EC_EXEC_AUTO / EC_EXEC_COMPILED;
 * with EC_EXEC_DENSE or EC_EXEC_INTERP every program runs on that tier),
 * and upload the stripe descriptors and work-item list (device memory owned
 * by the batch).  Block pointers are captured; the buffers must stay valid
 * while the batch runs. */
ec_status ec_batch_create(const ec_job *jobs, int n_jobs, int executor, ec_batch **out);
/* Enqueue the batch on `stream`: one persistent launch per module plus at
 * most one launch for the programs without a module (the dense bitmatrix
 * executor; the interpreter in batches created with EC_EXEC_INTERP).
 * Allocates nothing (capturable).  Large
 * launches split their work items into one contiguous range per SM; the
 * CTAs of an SM start on its range and then help with the others, so each
 * SM runs few distinct programs at a time. */
ec_status ec_batch_run(ec_batch *batch, void *stream);
/* The batch's own status word: *status = 0 or EC_ETIMEOUT when a bounded
 * wait of one of its runs gave up since the last reset (that run's outputs
 * are incomplete).  Synchronises the current device first; reset != 0
 * clears the word.  The device's word (ec_device_status) is set as well. */
ec_status ec_batch_status(ec_batch *batch, int *status, int reset);
ec_status ec_batch_info_get(const ec_batch *batch, ec_batch_info *out);
void ec_batch_destroy(ec_batch *batch);
/* create + run + synchronise + destroy; EC_ETIMEOUT when a bounded wait of
 * the run gave up. */
ec_status ec_run_batch(const ec_job *jobs, int n_jobs, void *stream);

/* ------------------------------------------------------------------ serving
 * Continuous batching of encode/decode requests.  Jobs submitted from any
 * thread are admitted while the block bytes of admitted, unfinished
 * requests stay within hbm_budget (else EC_EBUSY: retry later).  A
 * scheduler thread forms a batch from every request that arrived while
 * earlier batches were on the GPU and launches it on one of `slots`
 * streams, so that batches overlap on the device; completion events
 * timestamp each request.  Job pointers are captured at submission; the
 * buffers must stay valid until the ticket is returned by ec_server_poll. */
typedef struct ec_server ec_server;

typedef struct {
  size_t hbm_budget;     /* bytes of request blocks admitted at once (0 = 32 GiB) */
  int max_batch;         /* requests per batch (0 = 512)                          */
  int slots;             /* batches in flight on separate streams (0 = 4)         */
  int idle_spin_us;      /* after its last work the scheduler keeps polling for
                            this long before it sleeps on a condition variable
                            (0 = 1000 us; < 0 = sleep at once).  Polling costs
                            one host core and spares each request the wake-up */
  int no_background_compile; /* nonzero: a request whose program has no compiled
                            kernel always runs on the dense bitmatrix
                            executor.  Default: it runs there while a background
                            thread compiles the program, and later requests
                            use the compiled kernel.  Plans used with a server
                            must then stay alive until ec_server_destroy
                            returns                                            */
} ec_server_opts;

typedef struct {
  long long submitted, completed, rejected, failed;  /* completed: tickets returned,
                                      failed ones included; failed: returned with
                                      a status other than EC_OK                 */
  long long batches, max_batch_seen;
  long long bytes_in, bytes_out;   /* block bytes read / written by completed requests */
  long long admitted_bytes;        /* currently admitted                             */
  long long pending;               /* admitted, not yet launched                     */
  int slots_busy;
  long long compiled_in_background; /* programs compiled by the background thread   */
  long long cancelled;             /* requests dropped by ec_server_cancel           */
} ec_server_stats;

ec_status ec_server_create(const ec_server_opts *opts, ec_server **out);
/* Build and compile, before serving, the encoder and every decoder of up to
 * max_erasures erasures of `plan`, so that no request waits for planning. */
ec_status ec_server_warm(ec_server *server, ec_plan *plan, int max_erasures);
ec_status ec_server_submit(ec_server *server, const ec_job *job, uint64_t *ticket);
/* Cancel a request that is still waiting for a batch: it is dropped, its
 * admitted bytes are returned and its ticket never completes (EC_OK).
 * EC_EBUSY when it is already on the GPU or done, EC_EINVAL for a ticket
 * the server never issued. */
ec_status ec_server_cancel(ec_server *server, uint64_t ticket);
/* Up to max completed tickets (and their latency from submission, in
 * microseconds) since the last call; *n_done receives the count.  The
 * arrays are filled in every case; the return value is the status of the
 * first returned request that failed (EC_OK when none did). */
ec_status ec_server_poll(ec_server *server, uint64_t *tickets, double *latency_us, int max,
                         int *n_done);
/* Same, with each request's own status in status[i] (NULL: not wanted):
 * EC_OK; EC_ETIMEOUT when a bounded wait of its batch gave up (each slot has
 * its own status word, cleared at every dispatch); EC_ENOMEM, EC_ENOTSUP or
 * EC_ECUDA when its batch could not be launched.  A failed request's
 * outputs are incomplete; it is returned only after every kernel of its
 * batch has finished, and its admitted bytes are released.  Returns EC_OK
 * unless the CUDA context failed. */
ec_status ec_server_poll_ex(ec_server *server, uint64_t *tickets, double *latency_us, int *status,
                            int max, int *n_done);
ec_status ec_server_stats_get(ec_server *server, ec_server_stats *out);
/* Finish every admitted request, then free the server. */
void ec_server_destroy(ec_server *server);

/* Device status word written by kernels whose bounded waits gave up:
 * *status = 0 (ok) or EC_ETIMEOUT.  reset != 0 clears it.  Synchronises the
 * current device.  Also reads (and with reset clears) the status word that
 * ec_encode_noalloc's kernels write in its static scratch array. */
ec_status ec_device_status(int *status, int reset);

/* Diagnostics: launch a one-thread kernel that waits, with the same bounded
 * wait the pipelines use (about 2 s), on a barrier nothing completes.  The
 * wait gives up, the kernel records EC_ETIMEOUT in the status word read by
 * ec_device_status and returns; the context stays usable.  The paper has
 * no counterpart; this checks the failure path without faulting the GPU. */
ec_status ec_selftest_wait_timeout(void *stream);

/* Host check of an interpreter instruction stream (the format of
 * ec_plan_program): every statement well formed, operand ids below
 * n_in + n_slots, slots written before they are read, output strip ids
 * below n_out.  EC_OK, or EC_EINVAL with the first problem and its word
 * offset in ec_last_error.  The planner runs the same check on every
 * program it builds. */
ec_status ec_program_check(const uint16_t *code, size_t len, int n_in, int n_out, int n_slots);

/* Fault injection for tests: the n-th device or pinned-host allocation
 * made by the library from now on fails as if memory ran out (the call
 * that makes it returns EC_ENOMEM after freeing what it had allocated);
 * n = 0 clears it.  No GPU fault is involved.  The paper has no
 * counterpart. */
ec_status ec_debug_fail_alloc(int n);

/* Fault injection for tests: each of the next n calls of ec_batch_run,
 * serving dispatches and ec_encode_noalloc first enqueues, on its stream,
 * the bounded-wait self-test (ec_selftest_wait_timeout) aimed at the status
 * words that call's kernels use, so it reports EC_ETIMEOUT as if one of its
 * waits had given up (the real work still runs).  n = 0 clears it.  No GPU
 * fault is involved.  The paper has no counterpart. */
ec_status ec_debug_inject_timeout(int n);

/* Thread-local message of the last failure ("" if none). */
const char *ec_last_error(void);

/* Library version string. */
const char *ec_version(void);

/* ---------------------------------------------------------------- inputs
 * Fill n bytes at device pointer dst with bytes [offset, offset+n) of the
 * SplitMix64 stream `seed` (Steele, Lea and Flood 2014, counter form:
 * byte b is byte b%8 of mix(seed + (b/8 + 1) * 0x9E3779B97F4A7C15)).
 * Synthetic input generation only; not part of the coding method. */
ec_status ec_synth_fill(uint8_t *dst, size_t n, uint64_t seed, uint64_t offset, void *stream);

/* --------------------------------------------------- straight-line programs
 * Host-only access to the optimiser, for inspection and tests. */
typedef struct ec_slp ec_slp;

/* Parse the text form:  "const a b c" / "v = a b" / "ret v ..." lines. */
ec_status ec_slp_parse(const char *text, ec_slp **out);
/* Program of the bitmatrix of a rows x cols GF(2^8) matrix.  form 0: one
 * statement per row; form 1: binary left-to-right chains.  Rows are emitted
 * block by block, bit 7 down to bit 0 within a block. */
ec_status ec_slp_from_matrix(int rows, int cols, const uint8_t *A, int form, ec_slp **out);
ec_status ec_slp_repair(const ec_slp *in, int xor_cancel, ec_slp **out);
ec_status ec_slp_fuse(const ec_slp *in, int cancel_pairs, ec_slp **out);
/* kind: EC_SCHED_DFS or EC_SCHED_GREEDY (cap = cache capacity).  The result
 * is the pebble program of the paper's game (goals keep their pebbles). */
ec_status ec_slp_schedule(const ec_slp *in, int kind, int cap, ec_slp **out);
ec_status ec_slp_stats_get(const ec_slp *p, ec_slp_stats *out);
/* IOcost(P, cap) and CCap(P) of the abstract LRU cache (Sec. 6.2). */
long ec_slp_iocost(const ec_slp *p, int cap);
int ec_slp_ccap(const ec_slp *p);
/* *eq = 1 when both programs return the same sets of constants (Sec. 4.1). */
ec_status ec_slp_equivalent(const ec_slp *a, const ec_slp *b, int *eq);
/* Text form into buf (NUL-terminated); *need receives the length + 1. */
ec_status ec_slp_to_text(const ec_slp *p, char *buf, size_t len, size_t *need);
void ec_slp_destroy(ec_slp *p);

#ifdef __cplusplus
}
#endif
#endif /* XOREC_H */
