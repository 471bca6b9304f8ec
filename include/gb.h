/*
 * gb.h -- C ABI of the GB300 interval branch-and-bound global minimiser.
 *
 * The library encloses the global minimum of f(x) subject to l <= x <= u
 * (the problem of Eqs. 1-2 of Zhang, Shan and Cagan, "Global optimization
 * tailored for graphics processing units") with outward-rounded interval
 * arithmetic on the GPU (section 2.1, Eqs. 3-6).  Each generation selects a
 * batch of boxes with the smallest lower bounds (section 3.1, "select"),
 * splits each on the coordinates of its variable-cycling block (section 3.2,
 * Eqs. 7-11), samples f at every child's midpoint to lower the incumbent
 * upper bound GUB (section 3.1, "sample"), evaluates F(X) and the interval
 * gradient of every child, rules children out by the cut-off test
 * (LB > GUB) and the first-order test (section 3.1, "partition and rule
 * out"), and inserts the survivors into a pool kept in GPU memory.  The solve
 * stops when every remaining box has a lower bound within tol_f of GUB.
 *
 * Conventions for every entry point:
 *  - No call aborts, throws or exits; failures return a gb_status and
 *    gb_last_error() describes the most recent failure on the calling thread.
 *  - Pointers named h_* are host memory, d_* are device memory of the
 *    problem's CUDA device; "stream" is a cudaStream_t (NULL = legacy
 *    default stream).
 *  - Inputs are copied at the call; the caller keeps ownership of them.
 *  - Results returned in a gb_result are owned by the library until
 *    gb_free_result().
 *  - There is no CPU fallback: without a usable CUDA device the calls that
 *    need one return GB_E_CUDA.
 */
#ifndef GB_H
#define GB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gb_status {
    GB_OK = 0,
    GB_E_INVALID = 1,   /* malformed problem, options or arguments */
    GB_E_OOM = 2,       /* device or host allocation failed */
    GB_E_CAPACITY = 3,  /* box pool full; the returned enclosure is still rigorous */
    GB_E_LIMIT = 4,     /* generation limit reached; enclosure still rigorous */
    GB_E_TIMEOUT = 5,   /* a bounded device wait gave up */
    GB_E_CUDA = 6,      /* CUDA runtime error or no device */
    GB_E_BUSY = 7       /* serving: request not finished / no slot free */
} gb_status;

/* ---------------------------------------------------------------------- */
/* Objective: expression DAG (input format, 32-byte nodes)                 */
/* ---------------------------------------------------------------------- */
/* Node operators.  Nodes are topologically ordered (operand index < node
 * index).  ISUM(a = template root, b = first, c = end, d = step) is the sum
 * over i in {b, b+d, ...} < c of the template sub-DAG rooted at a, and
 * IPROD (same fields) the product (the Griewank, Styblinski and Zabinsky
 * functions of the paper's SI Appendix A; IPROD problems run on the
 * interpreter kernels, eval_mode 0 or 1).  In a template
 * IDX_VAR(b = offset) stands for x[i+offset] and IDX_COEF(a = table,
 * b = offset) for coef_tables[a][i+offset].  CONST(v) is the exact double v;
 * PI and EULER are the constants pi and e, enclosed by adjacent doubles;
 * SCALE(a, v) multiplies node a by the exact double v.  STEP(a) is the unit
 * step H(a) = 1 for a >= 0, 0 for a < 0, for discontinuous objectives (SI
 * Appendix F); a box that holds the jump gets an unbounded partial through
 * it, so the first-order test never rules it out.  Template nodes may
 * not use VAR, ISUM or IPROD; outer nodes may not use IDX_VAR or IDX_COEF. */
enum {
    GB_OP_CONST = 0, GB_OP_PI = 1, GB_OP_EULER = 2, GB_OP_VAR = 3,
    GB_OP_IDX_VAR = 4, GB_OP_IDX_COEF = 5, GB_OP_ADD = 6, GB_OP_SUB = 7,
    GB_OP_MUL = 8, GB_OP_DIV = 9, GB_OP_NEG = 10, GB_OP_SQR = 11,
    GB_OP_SQRT = 12, GB_OP_EXP = 13, GB_OP_SIN = 14, GB_OP_COS = 15,
    GB_OP_SCALE = 16, GB_OP_ISUM = 17, GB_OP_IPROD = 18, GB_OP_STEP = 19
};

typedef struct gb_node {
    int32_t op;   /* GB_OP_* */
    int32_t a;    /* operand 1 | VAR coordinate | IDX_COEF table | ISUM / IPROD template root */
    int32_t b;    /* operand 2 | IDX_VAR / IDX_COEF offset | ISUM / IPROD first index */
    int32_t c;    /* ISUM / IPROD end index (exclusive) */
    int32_t d;    /* ISUM / IPROD step (>= 1) */
    int32_t pad;  /* must be 0 */
    double v;     /* CONST value | SCALE factor */
} gb_node;

/* ---------------------------------------------------------------------- */
/* Options                                                                 */
/* ---------------------------------------------------------------------- */
typedef struct gb_options {
    double tol_f;             /* target width of [fmin_lo, fmin_hi] (<= 0: use the tol argument) */
    double tol_x;             /* a box narrower than tol_x in every coordinate is final (0 = off) */
    int32_t block;            /* cycling block size B, section 3.2 (0: min(n, 10)) */
    int32_t split_m;          /* pieces per split coordinate, 2 or 4 (0: 2) */
    int32_t split_d;          /* coordinates split per generation, 1..B, m^d <= 2^20 (0: B, capped so m^d <= 4096) */
    int32_t fp32_prefilter;   /* 1: FP32 directed-rounding pass before FP64 */
    int64_t max_generations;  /* 0: 10^9 */
    int64_t max_children;     /* children evaluated per generation (0: 1 << 22) */
    int64_t max_boxes;        /* pool capacity in boxes (0: from pool_bytes) */
    size_t pool_bytes;        /* device memory budget for the pool (0: 16 GiB) */
    int32_t device;           /* CUDA device ordinal */
    int32_t eval_mode;        /* child evaluation: 0 auto (term tables when m^d >= 16 and they fit),
                                 1 bytecode interpreter, 2 term tables when they fit (one child per warp
                                 when a generation has fewer than 2^16 children, else per thread),
                                 3 / 4 term tables with one child per thread / per warp; results are
                                 identical */
    int32_t gens_per_sync;    /* <= 1: the host reads the state after every generation (per-kernel timing);
                                 G > 1: generations run as replays of a captured CUDA graph, G between
                                 state reads (the search is the same) */
    int32_t pool_mode;        /* box storage (the list L of section 3.2): 0 auto (block records when
                                 n >= 128, a child replaces at most a quarter of the blocks and neither
                                 samples nor mono_all is set), 1 one dense row of n coordinates per box,
                                 2 block records shared between a box and its children (also with
                                 samples / mono_all: the way to hold the paper's procedure's 10^7-region
                                 lists); results are identical */
    int32_t samples;          /* GUB samples per box: 0 the midpoint; S in 1..64 the S interior points
                                 j / (S + 1) of its diagonal (the paper takes 10, section 4); S > 0 needs
                                 eval_mode 0 or 1 (bytecode interpreter) */
    int64_t max_records;      /* block records: record capacity (0: 4 * nrec * boxes + blocks, nrec = blocks
                                 a child replaces); unreferenced records are collected when new ones do not fit */
    int32_t mono_all;         /* 1: first-order test on every coordinate (the paper's rule, section 3.1)
                                 instead of the active block; needs eval_mode 0 or 1 */
    int32_t pad;
} gb_options;

/* Fills *opt with the defaults documented above. */
void gb_default_options(gb_options* opt);

/* ---------------------------------------------------------------------- */
/* Problems and solves                                                     */
/* ---------------------------------------------------------------------- */
typedef struct gb_problem gb_problem;

/* Creates a problem: minimise node `root` of h_dag[0..n_nodes) over the box
 * l <= x <= u (Eqs. 1-2; l < u finite, u - l finite), with coefficient
 * tables h_tables[t][0..h_table_lens[t]).  tol is the enclosure width target
 * (overridden by opt->tol_f when > 0).  opt may be NULL for the defaults.
 * The DAG is compiled to device bytecode and copied to the device together
 * with the tables.  Returns GB_E_INVALID for a malformed DAG or bounds,
 * GB_E_CUDA without a device, GB_E_OOM on allocation failure.  *out is set
 * only on GB_OK and must be released with gb_destroy_problem(). */
gb_status gb_create_problem(const gb_node* h_dag, int32_t n_nodes, int32_t root,
                            const double* const* h_tables, const int64_t* h_table_lens,
                            int32_t n_tables, int32_t n, const double* l, const double* u,
                            double tol, const gb_options* opt, gb_problem** out);

/* Per-generation counters of a solve (one row per generation). */
typedef struct gb_gen_stat {
    int64_t parents;   /* boxes selected and split */
    int64_t children;  /* children evaluated */
    int64_t kept32;    /* children kept by the FP32 pass (= children without it) */
    int64_t kept;      /* children inserted into the pool */
    int64_t pool;      /* pool size after the generation */
    double gub;        /* incumbent upper bound after the generation */
} gb_gen_stat;

typedef struct gb_result {
    double fmin_lo, fmin_hi;  /* rigorous enclosure [GLB, GUB] of min f */
    int64_t n_boxes;          /* boxes that may contain a global minimiser */
    int32_t n;                /* problem dimension */
    int32_t status;           /* gb_status of the solve */
    double* box_lo;           /* n_boxes x n, row-major, host (NULL from gb_solve_device) */
    double* box_hi;
    double* box_flo;          /* lower bound of f on each box */
    int64_t generations;
    int64_t box_evals_fp32;   /* children evaluated in FP32 (F and gradient) */
    int64_t box_evals_fp64;   /* children evaluated in FP64 (F and gradient) */
    int64_t mid_evals;        /* FP64 midpoint samples */
    double solve_ms;          /* wall time of the solve on the host clock */
    double device_ms;         /* CUDA-event time from the first to the last launch */
    double eval64_ms;         /* CUDA-event time of the child evaluation: per-parent term tables, FP32 pass
                                 and FP64 kernels (with gens_per_sync <= 1) */
    double eval32_ms;         /* CUDA-event time inside the FP32 evaluation kernels (part of eval64_ms) */
    int64_t eval64_launches;
    int64_t eval32_launches;
    int64_t kernel_launches;  /* kernels the library launched for this solve */
    int64_t ops64;            /* directed-rounding FP64 operations executed by the evaluation (tables, children) */
    int64_t ops32;            /* directed-rounding FP32 operations executed by the evaluation (tables, children) */
    double queue_ms;          /* serving: submit -> admission (host clock); 0 for gb_solve */
    double latency_ms;        /* serving: submit -> result ready (host clock); 0 for gb_solve */
    int32_t pool_mode;        /* box storage used: 1 dense rows, 2 block records */
    int32_t pad;
    int64_t record_gcs;       /* block records: collections run */
    int64_t n_trace;
    gb_gen_stat* trace;       /* n_trace rows, host */
} gb_result;

/* Solves the problem (blocking).  Copies the enclosure, the surviving boxes
 * and the per-generation trace to host memory in *out.  On GB_E_CAPACITY or
 * GB_E_LIMIT the enclosure and boxes returned are still rigorous.  The
 * problem can be solved again; each solve starts from the whole domain. */
gb_status gb_solve(gb_problem* prob, gb_result* out);

/* Same solve, leaving the surviving boxes on the device (box_lo/box_hi/
 * box_flo are NULL in *out).  Used to time the device path alone. */
gb_status gb_solve_device(gb_problem* prob, gb_result* out);

/* Releases the host arrays of a result (safe on a zeroed result). */
void gb_free_result(gb_result* res);

/* ---------------------------------------------------------------------- */
/* Checkpoint and resume of the region list (section 3.1's list L)          */
/* ---------------------------------------------------------------------- */
/* The pool a solve left behind: every region, active or final, in pool
 * order (the order the best-first selection breaks ties by), with its lower
 * bound, its cycling word and the incumbent GUB.  Host arrays, owned by the
 * library until gb_free_snapshot. */
typedef struct gb_snapshot {
    int32_t n;                /* problem dimension */
    int32_t block;            /* cycling block size of the problem it was taken from */
    int64_t count;            /* regions */
    double* lo;               /* count x n, row-major */
    double* hi;
    double* flo;              /* lower bound of f on each region (as the pool holds it) */
    int32_t* cyc;             /* next coordinate to split; bit 31 marks a final region (all widths < tol_x) */
    double gub;               /* incumbent upper bound of the minimum */
    int64_t generations;      /* generations run to reach this pool, over every call */
} gb_snapshot;

/* Takes the pool left by the last gb_solve / gb_solve_device /
 * gb_solve_resume on prob (whatever its status: a solve stopped by
 * max_generations or by GB_E_CAPACITY leaves a valid pool).
 * GB_E_INVALID if no solve has run, GB_E_BUSY while one runs. */
gb_status gb_snapshot_take(gb_problem* prob, gb_snapshot* out);

/* Continues the branch and bound from a snapshot instead of the domain:
 * the regions enter the pool in snapshot order with their lower bounds and
 * cycling words, the incumbent is the snapshot's GUB, and the per-region
 * cached sums are recomputed.  prob must have the snapshot's n; its other
 * options may differ (a larger pool, another generation limit or device).
 * With the same block, split and selection options the run continues
 * exactly as the uninterrupted solve would: the generations of the resumed
 * call follow those of the snapshot.  out->generations counts this call.
 * Needs dense rows (pool_mode 1).  GB_E_INVALID on a mismatched or
 * malformed snapshot (regions outside the bounds, lo > hi, a cycling word
 * out of range, a NaN bound), GB_E_CAPACITY if the regions do not fit. */
gb_status gb_solve_resume(gb_problem* prob, const gb_snapshot* snap, gb_result* out);

/* Releases the host arrays of a snapshot (safe on a zeroed one). */
void gb_free_snapshot(gb_snapshot* snap);

/* Releases the problem and all its device memory. */
void gb_destroy_problem(gb_problem* prob);

const char* gb_status_str(gb_status s);
const char* gb_last_error(void);

/* ---------------------------------------------------------------------- */
/* Serving: continuous batching of many problems on one GPU                */
/* ---------------------------------------------------------------------- */
/* A server runs independent minimisation requests concurrently on one GPU
 * (the paper solves one problem at a time; this is the serving form of the
 * same method).  Requests are admitted in arrival order while the device
 * memory they reserve (opt->pool_bytes, or budget / max_active when 0) fits
 * the budget and fewer than max_active are running; each admitted request
 * runs its generations on its own stream, and the server advances whichever
 * request's previous generation has finished, so the requests' kernels
 * overlap on the device.  Finished requests free their memory and slot for
 * the queued ones.  A request's result does not depend on the others.
 * Fused mode (gb_server_set_fused): the requests whose children are
 * evaluated by the term-table FP32-then-FP64 kernel advance in steps of 4
 * generations: every such request whose previous step has finished joins
 * the next one, and each generation of a step evaluates the children of all
 * its requests in one persistent launch (each warp takes a few children of
 * one request, with that request's program, tables and incumbent); the
 * other requests advance on their own as above.  Results are the same in
 * both modes. */
typedef struct gb_server gb_server;

/* Starts a server (and its worker thread) on `device`.  pool_budget_bytes
 * bounds the device memory reserved by running requests.  Returns
 * GB_E_INVALID for a zero budget or max_active < 1, GB_E_CUDA without the
 * device. */
gb_status gb_server_create(size_t pool_budget_bytes, int32_t device, int32_t max_active, gb_server** out);

/* fused = 1: one fused child-evaluation launch per generation over the
 * eligible requests of a step; 0 (default): every request advances on its
 * own, 4 generations per CUDA-graph replay.  May be changed at any time; it
 * applies from the next step.  GB_E_INVALID for a NULL server. */
gb_status gb_server_set_fused(gb_server* srv, int32_t fused);

/* Queues a request (same arguments as gb_create_problem; everything is
 * copied) and returns at once with its id.  Never blocks on the GPU.
 * GB_E_BUSY if the server is shutting down. */
gb_status gb_submit(gb_server* srv, const gb_node* h_dag, int32_t n_nodes, int32_t root,
                    const double* const* h_tables, const int64_t* h_table_lens, int32_t n_tables,
                    int32_t n, const double* l, const double* u, double tol, const gb_options* opt,
                    uint64_t* request_id);

/* GB_E_BUSY while the request is queued or running.  Once it has finished,
 * fills *out (host arrays owned by the caller from then on: release with
 * gb_free_result; queue_ms / latency_ms set), forgets the id and returns the
 * solve's status.  GB_E_INVALID for an unknown id. */
gb_status gb_poll(gb_server* srv, uint64_t request_id, gb_result* out);

/* Stops the worker, releases running requests and unclaimed results. */
gb_status gb_server_destroy(gb_server* srv);

/* ---------------------------------------------------------------------- */
/* Parity hook: evaluate given boxes from scratch                          */
/* ---------------------------------------------------------------------- */
/* For each of nbox boxes (d_lo, d_hi: nbox x n row-major, device) computes
 * F(X) (d_F: nbox x 2), the FP64 midpoint sample F([m, m]) with
 * m = RN(0.5 lo + 0.5 hi) (d_Fmid: nbox x 2), the interval partials of the
 * coordinates of cycling block `block_index` (d_G: nbox x B x 2, tail of a
 * short last block untouched) and the first-order verdict (d_mono: 1 if
 * some tested partial excludes 0 away from the domain edge, section 3.1).
 * fp32 = 1 evaluates F and G in FP32 directed rounding (the box widened
 * outward to floats); Fmid is always FP64.  Runs on `stream`; no sync. */
gb_status gb_eval_boxes(gb_problem* prob, const double* d_lo, const double* d_hi,
                        int64_t nbox, int32_t block_index, int32_t fp32, double* d_F,
                        double* d_Fmid, double* d_G, int32_t* d_mono, void* stream);

/* gb_eval_boxes without any device allocation, for callers that cannot
 * allocate device memory while they run (for example a serving process that
 * has already handed all free device memory to its own pool, or a
 * latency-critical thread that must not wait on the device allocator).
 * Same arguments and results as gb_eval_boxes.  The paper has no counterpart
 * of this entry point.
 *  - The FP32 copy of the boxes that fp32 = 1 needs is kept in a fixed array
 *    inside the library instead of a per-call buffer: at most 2^20
 *    coordinates (nbox * n <= 1048576) per FP32 call; larger FP32 calls
 *    return GB_E_INVALID with a message.  fp32 = 0 needs no scratch and has
 *    no size limit.  The array (8 MiB) is held on every GPU that loads the
 *    library until the process exits.
 *  - The first FP32 call on a device looks up the array's device address
 *    with that device current (a failed lookup is retried by the next call);
 *    make that first call before any stream capture.  The caller's current
 *    device is left as it was.
 *  - Every call shares the one array; each call writes the part it uses
 *    before reading it, so no clearing is needed, but calls whose work
 *    overlaps on the GPU (unordered streams or threads) race. */
gb_status gb_eval_boxes_noalloc(gb_problem* prob, const double* d_lo, const double* d_hi,
                                int64_t nbox, int32_t block_index, int32_t fp32, double* d_F,
                                double* d_Fmid, double* d_G, int32_t* d_mono, void* stream);

/* Block size B, number of blocks and the static count of directed-rounding
 * floating-point operations of one F+gradient child evaluation and one
 * midpoint sample (FP64), as compiled. */
gb_status gb_problem_info(const gb_problem* prob, int32_t* block, int32_t* n_blocks,
                          int64_t* ops_eval, int64_t* ops_mid);

/* ---------------------------------------------------------------------- */
/* Measurement helper (the paper has no counterpart)                        */
/* ---------------------------------------------------------------------- */
/* Throughput of directed-rounding arithmetic on `device`, for roofline
 * denominators: which = 0 times FP64 __dadd_rd/__dmul_ru chains, which = 1
 * the FP32 __fadd_rd/__fmul_ru forms.  Runs a register-resident kernel on
 * all SMs and returns operations per second in *ops_per_s and the kernel's
 * CUDA-event time in *ms.  Blocking. */
gb_status gb_measure_peak(int32_t device, int32_t which, double* ops_per_s, double* ms);

/* ---------------------------------------------------------------------- */
/* Autotuner of the batching layer (the paper fixes m = 4, d = 10, §4)      */
/* ---------------------------------------------------------------------- */
/* Times complete solves of the problem (arguments as in gb_create_problem)
 * under candidate settings of the bisection fan-out (split_m in {2, 4},
 * split_d in {B, ceil(B/2)} with m^d <= 2^20), the parents per generation
 * (max_children = 1 or 4 times m^d) and the child-kernel shape (eval_mode 3:
 * one child per thread, 4: one child per warp, when term tables are used),
 * starting from *base (NULL: defaults; its block, tolerances, precision,
 * pool and device are kept), and writes the fastest setting to *best and its
 * solve time (ms, host clock, second of two solves) to *best_ms.  Every
 * candidate is a rigorous solve; only the time differs.  Candidates ending
 * with GB_E_CAPACITY or GB_E_LIMIT are skipped; candidates are tried while
 * the elapsed time is below budget_ms (at least one is always tried).
 * Returns GB_E_LIMIT if no candidate completed.  Blocking; allocates and
 * frees one problem per candidate. */
gb_status gb_autotune(const gb_node* dag, int32_t n_nodes, int32_t root, const double* const* tables,
                      const int64_t* table_lens, int32_t n_tables, int32_t n, const double* l, const double* u,
                      double tol, const gb_options* base, double budget_ms, gb_options* best, double* best_ms);

#ifdef __cplusplus
}
#endif

#endif /* GB_H */
