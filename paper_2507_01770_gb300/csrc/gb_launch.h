// Launch wrappers of the solver kernels (gb_kernels.cu), used by gb_api.cu.
#pragma once
#include <cuda_runtime.h>

#include "gb_internal.h"

#define GB_FINAL_BIT 0x80000000u

// Box store: one slot per box, slot-major rows.
struct GbPool {
    double* lo64;     // [cap][n]
    double* hi64;
    float* lo32;      // [cap][n] outward float shadow (FP32 prefilter only)
    float* hi32;
    double2* gsum;    // [cap][NG] cached group sums of F (FP64)
    double2* gmid;    // [cap][NG] cached group sums at the box midpoint (FP64)
    float2* gsum32;   // [cap][NG] cached group sums of F (FP32 prefilter only)
    unsigned* freel;  // [cap] free slots
    double2* gsamp;   // [cap][S][NG] cached group sums at the S diagonal samples (dense rows, samples > 0)
    double2* gdp;     // [cap][n_sum][n] cached coordinate partial sums D (dense rows, mono_all)
    double2* rgsamp;  // [S][R][GPB] the owned groups' sums at the S diagonal samples (records, samples > 0)
    double2* rgdp;    // [R][n_sum][B] coordinate partial sums D of the record's block (records, mono_all,
                      // templates confined to one coordinate)
    int n, NG, fp32, S;
    // block-record mode (recs = 1): a box is a row of nb record ids; record q
    // holds block coordinates [q*B, q*B + B) and the cached sums of the groups
    // its block owns [q*GPB, q*GPB + GPB).  lo64..gsum32 above are unused.
    int recs, nb, B, GPB, nrec;
    unsigned* rid;    // [cap][nb]
    double* rlo;      // [R][B]
    double* rhi;
    float* rlo32;     // [R][B] (FP32 prefilter only)
    float* rhi32;
    double2* rgsum;   // [R][GPB]
    double2* rgmid;
    float2* rgsum32;
    unsigned* rfree;  // [R] free records
    unsigned* rmark;  // [R] collection number that last found the record referenced
    unsigned char* rwide;  // [R] 1: some coordinate of the record is at least tol_x wide
    int* swide;       // [cap] records of the box with rwide = 1 (0: the box is final)
    long long R;      // record capacity
};

// Ordered list of pool entries (the best-first list; bit 31 of cyc = final).
struct GbEntries {
    double* flo;
    unsigned* slot;
    int* cyc;
};

struct GbParents {
    unsigned* slot;
    int* cyc;
    double* flo;
    int4* info;       // c0 (first split coordinate), dd (coordinates split), block, next cyc
    double* bnd;      // [K][dmax][m+1] piece boundaries
    float* bnd_rd;    // boundaries rounded down / up to float
    float* bnd_ru;
};

struct GbChildren {
    double* flo;
    unsigned char* flag;
    unsigned char* flag32;
    unsigned* list32;
    unsigned* surv;
};

struct GbSplit {
    int m, mshift, d, flog2;   // pieces, log2(pieces), coordinates split, log2(fan-out)
    int dmax;                  // boundary table stride (coordinates)
};

// Per-parent term tables (rows indexed by parent * max_rows + row) and the
// parent's group-sum trees (nodes indexed by parent * tree_nodes + node).
struct GbTabs {
    double2* tv64;    // term value over the box
    double2* tm64;    // term value at the box midpoint
    double2* tl64;    // leaf adjoints, max_leaves per row
    float2* tv32;     // FP32 term value (FP32 prefilter only)
    float2* tl32;     // FP32 leaf adjoints
    double2* nf64;    // group tree of the parent's cached sums: F
    double2* nm64;    // midpoint
    float2* nf32;     // FP32
    double2* td64;    // per (coordinate, sum) sums of leaf adjoints by digit combination
    float2* td32;     // FP32
    double2* ts64;    // term-tree segment sums by digit combination: F
    double2* tsm64;   // midpoint
    float2* ts32;     // FP32
    int max_rows, max_leaves, tree_nodes, max_drows, max_srows;
    int warp;         // child kernels: 1 one child per warp, 0 one child per thread
    int max_sum_nodes;   // nodes of the largest sum's group tree
    int tree_smem;       // 1: k_ptab builds the group trees in shared memory (they fit)
    // one child per warp: every child's sums and dirty group values, computed
    // before the child kernel by k_child_sums (null otherwise)
    double2* cs64;    // [Cmax][n_sum] F
    double2* csm64;   // [Cmax][n_sum] midpoint
    float2* cs32;     // [Cmax][n_sum] FP32
    double2* cg64;    // [Cmax][GB_CG] dirty group values, slot k * GB_TAB_MAX_DIRTY + (g - first dirty group)
    double2* cgm64;
    float2* cg32;
    // one child per warp, objectives whose sums all enter F with adjoint
    // [1, 1] and no coordinate of their own in the outer expression: the
    // first-order verdict of each block coordinate for every combination of
    // the digit bits its partial depends on (at most GB_MV_BITS of them), per
    // parent, written by k_child_sums (null otherwise)
    unsigned char* mv64;   // [K][B][1 << GB_MV_BITS]
    unsigned char* mv32;
    // with the verdict tables: each block coordinate's digit field in them
    // (first bit | bit count << 8; 0xffff: the coordinate has none), per
    // parent -- it depends on the parent's split alone
    unsigned short* mvb;   // [K][B]
    // one child per thread, objectives whose outer expression is one sum:
    // 1 when every block's dirty groups fit the register-resident walk (at
    // most GB_REG_DIRTY groups of fewer than 2^GB_REG_LEVELS terms each)
    int reg;
};
constexpr int GB_CG = GB_MAX_ISUM * GB_TAB_MAX_DIRTY;
constexpr int GB_MV_BITS = 6;
constexpr int GB_REG_DIRTY = 4;
constexpr int GB_REG_LEVELS = 5;

// scratch for the scans
struct GbScan {
    int* tile_cnt;     // [3][max_tiles] tile counts (pool partition: aggregates)
    int* tile_off;     // [3][max_tiles] tile offsets (pool partition: inclusive prefixes)
    unsigned* hist;    // [65536] radix-select histogram
    unsigned long long* tile_flag;   // [max_tiles] pool partition: epoch << 2 | 1 aggregate / 2 prefix published
    unsigned long long* stat_key;    // [GB_STAT_BLOCKS] per-block smallest active key (k_stats)
    long long* stat_pos;             // [GB_STAT_BLOCKS] its last pool position in that block
    int max_tiles;
};
constexpr int GB_STAT_BLOCKS = 4096;   // grid cap of k_stats

constexpr int GB_TILE = 1024;

// Constants of a problem's generations (kernel arguments that never change,
// so a generation's launches can be captured once and replayed).
struct GbGenConst {
    long long K;            // parents per generation
    int flog2;              // log2 of the fan-out
    int fp32;               // FP32 prefilter on
    long long max_gen;
    double tol_f, tol_x;
    gb_gen_stat* trace;     // device rows, one per generation
    long long trace_cap;
    int nrec;               // block records: new records per child (0: dense rows)
    long long R;            // block records: capacity
};

// Child kernels run one child per warp when a generation has few children
// (fewer than 2^16: one child per thread would leave most of the SMs idle),
// else one child per thread (eval_mode 3 / 4 force either).
inline bool gb_warp_per_child(long long Cmax) { return Cmax < (1LL << 16); }

cudaError_t gb_launch_root_init(const GbProg& P, const GbPool& pool, const GbEntries& E, double tol_x,
                                GbState* st, cudaStream_t s);
// Active count of the pool; count and GUB are read from the device state,
// max_count bounds the grid.
// Active count of the pool (read from the device state) for the next generation.
// par / pool non-null: at the end of a generation (free the parents, roll
// the counters forward first).
cudaError_t gb_launch_stats(const GbEntries& E, const GbGenConst& G, long long cap, const GbScan& sc, GbState* st,
                            cudaStream_t s, const GbParents* par = nullptr, const GbPool* pool = nullptr);
// Checkpoint: every entry of E[0, count) with its box (lo, hi: count x n), LB and cycling word.
cudaError_t gb_launch_snapshot(const GbEntries& E, long long count, const GbPool& pool, double* lo, double* hi,
                               double* flo, int* cyc, cudaStream_t s);
// Resume (dense rows): boxes to slots 0 .. count-1 with recomputed caches, entries in the given order, and
// the device state of a pool of `count` entries with incumbent gub.
cudaError_t gb_launch_resume(const GbProg& P, const GbPool& pool, const GbEntries& E, long long count,
                             const double* lo, const double* hi, const double* flo, const int* cyc, double gub,
                             GbState* st, cudaStream_t s);
// One generation: select, partition, prepare parents, (term tables), evaluate
// children (FP32 pass, compaction, FP64 pass), compact survivors,
// materialise, free parents, finish, and the active count of the new pool.
// Every size is read from the device state.  ev (4 events or null) brackets
// the FP64 and FP32 evaluation kernels.  Returns the kernels launched in
// *nlaunch.  part 1 stops before the child evaluation and part 2 starts
// after it (a fused evaluation over several problems goes between them).
// A second stream and two events of a problem: with one parent per
// generation and term tables, the parent's tables (k_ptab, k_ptab_d,
// k_child_sums) run on s2 beside the pool partition on the main stream (the
// parent is the pool entry k_stats found), joined before the child kernel.
struct GbFork {
    cudaStream_t s2;
    cudaEvent_t fork, join;
};
cudaError_t gb_launch_generation(const GbProg& P, const GbPool& pool, const GbEntries& E, const GbEntries& E_new,
                                 const GbParents& par, const GbChildren& ch, const GbSplit& sp, const GbScan& sc,
                                 const GbTabs* tabs, const GbGenConst& G, long long cap, long long Cmax,
                                 GbState* st, cudaStream_t s, cudaEvent_t* ev, long long* nlaunch, int part = 0,
                                 const GbFork* fork = nullptr);

// One problem of a fused child evaluation: the arguments of its
// k_eval3264_tabw launch (term tables, one child per warp, FP32 then FP64).
struct GbEvalDesc {
    GbProg P;
    GbPool pool;
    GbParents par;
    GbTabs Tb;
    GbChildren ch;
    GbSplit sp;
    GbState* st;
};
#define GB_BATCH_MAX 256   // problems per fused launch
// The children of every problem of D[0, nreq) in one persistent launch on s:
// each warp takes units of a few children of one problem in turn, with that
// problem's program, tables, incumbent and counters.  max_units (the units
// the step can hold at most) sizes the grid.
cudaError_t gb_launch_eval3264_batch(const GbEvalDesc* d_desc, int nreq, long long max_units, cudaStream_t s);
// Final output: entries with flo <= GUB, in pool order, gathered into rows.
cudaError_t gb_launch_output(const GbEntries& E, long long count, const GbPool& pool, double gub,
                             unsigned* list, double* out_lo, double* out_hi, double* out_flo,
                             GbState* st, const GbScan& sc, cudaStream_t s);
cudaError_t gb_launch_eval_boxes(const GbProg& P, const double* lo, const double* hi, float* scratch32,
                                 long long nbox, int blk, int fp32, double* F, double* Fmid, double* G,
                                 int* mono, cudaStream_t s);
cudaError_t gb_launch_peak(int which, int iters, int blocks, void* sink, cudaStream_t s);
long long gb_launches_so_far();
// Streaming multiprocessors of the current device (queried once per device).
int gb_sm_count();

// Programmatic dependent launch.  A kernel of the generation path starts with
// gb_grid_trigger() (its own dependent may be launched once all of its blocks
// have started) and gb_grid_wait() (it touches nothing before the kernels it
// depends on have completed and their writes are visible), so a launch with
// `pdl` can overlap its launch and block scheduling with the end of its
// predecessor in the stream.  A kernel launched without `pdl` waits as usual
// and the two calls return at once.  The overlap is off unless the
// environment sets GB_PDL=1: measured on GB300 it loses slightly (a C3
// generation 80.8 us with it, 79.1 us without; served solves 50.7/s with
// it, 53.4/s without), as the early blocks hold SM resources that the
// kernels of the other stream, or of other requests, could use.
// gb_pdl_thread(false) keeps it off for the calling thread's launches and
// graph captures whatever the environment (the serving worker).
bool gb_pdl_enabled();
void gb_pdl_thread(bool on);
template <typename... KArgs, typename... Args>
inline cudaError_t gb_launch_ex(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                                Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = (pdl && gb_pdl_enabled()) ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, ((KArgs)args)...);
}
extern "C" const GbProg* gb_internal_prog(const gb_problem* p, int* device, int* n, int* nb);
extern "C" gb_status gb_internal_fail(gb_status s, const char* msg);
// resumable solve (gb_api.cu), used by the serving loop (gb_server.cpp)
extern "C" gb_status solve_begin(gb_problem* p);
extern "C" int solve_advance(gb_problem* p, bool block);
extern "C" int solve_check(gb_problem* p, bool block);
extern "C" void solve_abort(gb_problem* p, gb_status st);   // ends the loop with st (solve_finish still runs)
// fused evaluation over several problems (gb_api.cu), used by the serving loop
struct GbBatchCtx;
extern "C" GbBatchCtx* batch_create(int device);
extern "C" void batch_destroy(GbBatchCtx* B);
extern "C" bool solve_fusable(const gb_problem* p);
extern "C" gb_status batch_generation(gb_problem* const* probs, int k, GbBatchCtx* B, int G);
extern "C" gb_status solve_finish(gb_problem* p, gb_result* out, bool copy_boxes);
extern "C" size_t gb_internal_device_bytes(const gb_problem* p);
// per-parent term tables (gb_kernels_tab.cu); sizes read from the device state
// Esel non-null: the single parent is pool entry st->sel_pos of *Esel (the
// partition may still be running).
cudaError_t gb_launch_ptab(const GbProg& P, const GbPool& pool, const GbParents& par, const GbTabs& T,
                           long long K, const GbSplit& sp, GbState* st, cudaStream_t s,
                           const GbEntries* Esel = nullptr);
cudaError_t gb_launch_eval64_tab(const GbProg& P, const GbPool& pool, const GbParents& par, const GbTabs& T,
                                 const GbChildren& ch, long long Cmax, const GbSplit& sp, bool from_list,
                                 GbState* st, cudaStream_t s);
// FP32 prefilter + FP64 evaluation fused, one child per warp (tables).
// Partial tables of every parent (after gb_launch_ptab).
// fixed: the generation has K parents for certain (do not read the count the partition writes).
cudaError_t gb_launch_ptab_d(const GbProg& P, const GbPool& pool, const GbParents& par, const GbTabs& T,
                             long long K, int B, GbState* st, cudaStream_t s, bool fixed = false);
// One child per warp: every child's sums and dirty group values (tables first).
cudaError_t gb_launch_child_sums(const GbProg& P, const GbPool& pool, const GbParents& par, const GbTabs& T,
                                 const GbSplit& sp, long long Cmax, int fp32, GbState* st, cudaStream_t s,
                                 bool fixed = false);
// cc non-null (at most 2^16 children): the kernel's last block also lists the survivors.
cudaError_t gb_launch_eval3264_tabw(const GbProg& P, const GbPool& pool, const GbParents& par, const GbTabs& T,
                                    const GbChildren& ch, long long Cmax, const GbSplit& sp, GbState* st,
                                    cudaStream_t s, const GbGenConst* cc = nullptr);
cudaError_t gb_launch_eval32_tab(const GbProg& P, const GbPool& pool, const GbParents& par, const GbTabs& T,
                                 const GbChildren& ch, long long Cmax, const GbSplit& sp, GbState* st,
                                 cudaStream_t s);
