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
    int n, NG, fp32;
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
    int max_rows, max_leaves, tree_nodes;
};

// scratch for the three-phase scans
struct GbScan {
    int* tile_cnt;     // [3][max_tiles]
    int* tile_off;     // [3][max_tiles]
    unsigned* hist;    // [65536] radix-select histogram
    int max_tiles;
};

constexpr int GB_TILE = 1024;

cudaError_t gb_launch_root_init(const GbProg& P, const GbPool& pool, const GbEntries& E, GbState* st,
                                cudaStream_t s);
// Active count of the pool; count and GUB are read from the device state,
// max_count bounds the grid.
cudaError_t gb_launch_stats(const GbEntries& E, long long max_count, double tol_f, GbState* st, cudaStream_t s);
cudaError_t gb_launch_select(const GbEntries& E, long long count, long long active, long long K,
                             double gub, double tol_f, GbState* st, const GbScan& sc, cudaStream_t s);
cudaError_t gb_launch_partition(const GbEntries& E, long long count, double gub, double tol_f,
                                const GbEntries& E_new, const GbParents& par, const GbPool& pool,
                                GbState* st, const GbScan& sc, cudaStream_t s);
cudaError_t gb_launch_prep(const GbProg& P, const GbPool& pool, const GbParents& par, long long npar,
                           const GbSplit& sp, GbState* st, cudaStream_t s);
cudaError_t gb_launch_eval64(const GbProg& P, const GbPool& pool, const GbParents& par,
                             const GbChildren& ch, long long nchildren, const GbSplit& sp, double gub_prev,
                             bool from_list, GbState* st, cudaStream_t s);
cudaError_t gb_launch_eval32(const GbProg& P, const GbPool& pool, const GbParents& par,
                             const GbChildren& ch, long long nchildren, const GbSplit& sp, double gub_prev,
                             GbState* st, cudaStream_t s);
// mode 0: list of FP32 survivors (flag32); mode 1: final survivors
// (flag && flo <= new GUB) with the capacity check.
cudaError_t gb_launch_compact_children(const GbChildren& ch, long long nchildren, int mode, GbState* st,
                                       const GbScan& sc, cudaStream_t s);
// tabs: the parents' term tables (null: dirty groups are re-interpreted)
cudaError_t gb_launch_materialize(const GbProg& P, const GbPool& pool, const GbParents& par,
                                  const GbChildren& ch, long long nchildren, const GbSplit& sp,
                                  const GbEntries& E_new, double tol_x, GbState* st, cudaStream_t s,
                                  const GbTabs* tabs);
cudaError_t gb_launch_finish(const GbParents& par, long long npar, const GbPool& pool,
                             const GbEntries& E_new, GbState* st, cudaStream_t s);
// Final output: entries with flo <= GUB, in pool order, gathered into rows.
cudaError_t gb_launch_output(const GbEntries& E, long long count, const GbPool& pool, double gub,
                             unsigned* list, double* out_lo, double* out_hi, double* out_flo,
                             GbState* st, const GbScan& sc, cudaStream_t s);
cudaError_t gb_launch_eval_boxes(const GbProg& P, const double* lo, const double* hi, float* scratch32,
                                 long long nbox, int blk, int fp32, double* F, double* Fmid, double* G,
                                 int* mono, cudaStream_t s);
cudaError_t gb_launch_peak(int which, int iters, int blocks, void* sink, cudaStream_t s);
long long gb_launches_so_far();
extern "C" const GbProg* gb_internal_prog(const gb_problem* p, int* device, int* n, int* nb);
extern "C" gb_status gb_internal_fail(gb_status s, const char* msg);
// resumable solve (gb_api.cu), used by the serving loop (gb_server.cpp)
extern "C" gb_status solve_begin(gb_problem* p);
extern "C" int solve_advance(gb_problem* p, bool block);
extern "C" gb_status solve_finish(gb_problem* p, gb_result* out, bool copy_boxes);
extern "C" size_t gb_internal_device_bytes(const gb_problem* p);
// per-parent term tables (gb_kernels_tab.cu)
cudaError_t gb_launch_ptab(const GbProg& P, const GbPool& pool, const GbParents& par, const GbTabs& T,
                           long long npar, const GbSplit& sp, cudaStream_t s);
cudaError_t gb_launch_eval64_tab(const GbProg& P, const GbPool& pool, const GbParents& par, const GbTabs& T,
                                 const GbChildren& ch, long long nchildren, const GbSplit& sp, double gub_prev,
                                 bool from_list, GbState* st, cudaStream_t s);
cudaError_t gb_launch_eval32_tab(const GbProg& P, const GbPool& pool, const GbParents& par, const GbTabs& T,
                                 const GbChildren& ch, long long nchildren, const GbSplit& sp, double gub_prev,
                                 GbState* st, cudaStream_t s);
long long gb_tab_launches_so_far();
