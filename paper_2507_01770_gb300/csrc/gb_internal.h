// Internal data structures of the library: the compiled device program of an
// objective and the device-side solver state.  Shared by the host compiler
// (gb_compile.cpp) and the CUDA kernels; not part of the public ABI.
#pragma once
#include <stdint.h>
#include <vector_types.h>

#include "../../include/gb.h"

#ifdef __CUDACC__
#define GB_HD __host__ __device__
#else
#define GB_HD
#endif

#ifdef __CUDACC__
// Programmatic dependent launch (see gb_launch_ex): let the stream's next
// kernel launch once every block of this one has started, and wait for the
// kernels this one depends on to complete before touching their results.
__device__ __forceinline__ void gb_grid_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void gb_grid_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
#endif

// Limits of the bytecode interpreter (registers live in thread-local arrays).
#define GB_MAX_TREGS 24   // nodes of one ISUM template
#define GB_MAX_OREGS 32   // nodes of the outer expression
#define GB_MAX_ISUM 6     // ISUM nodes per objective
#define GB_MAX_WIN 4      // IDX_VAR offset span + 1 per template
#define GB_MAX_SPLIT_D 20   // coordinates split per generation
#define GB_TAB_MAX_DIRTY 8  // dirty groups per sum for the table path
#define GB_TAB_MAX_ROWS 4096 // table rows per parent for the table path
#define GB_MAX_FAN_LOG2 20  // children per parent (m^d) at most 2^20

// Device opcodes of one instruction (registers are node slots).
enum GbDevOp : uint8_t {
    D_CONST = 0, D_PI, D_EULER, D_VAR, D_IVAR, D_COEF, D_ISUMV,
    D_ADD, D_SUB, D_MUL, D_DIV, D_NEG, D_SQR, D_SQRT, D_EXP, D_SIN, D_COS, D_SCALE, D_STEP
};

struct GbIns {
    uint8_t op;       // GbDevOp
    uint8_t dst;      // destination register
    uint8_t a, b;     // operand registers
    int32_t aux;      // VAR coordinate | IVAR offset | COEF table | ISUMV slot
    int32_t aux2;     // COEF offset
    float clo32;      // c rounded down to float
    float chi32;      // c rounded up to float
    int32_t pad;      // directed-op cost: forward (bits 0-7), reverse (bits 8-15)
    double c;         // CONST value | SCALE factor
};  // 32 bytes

// One ISUM (or IPROD) node: its template bytecode and the grouping of its terms.
// Terms are grouped into maximal runs with the same range of touched
// cycling blocks; the cached partial sums of a box are kept per group.
struct GbSum {
    int32_t ins0, nins;      // template instructions [ins0, ins0 + nins)
    int32_t first, step, count;  // index set {first + t * step : t < count}
    int32_t off_min, off_max, has_var;
    int32_t prod;            // 1: IPROD (product of the terms; empty product [1, 1])
    int32_t group0, ngroups; // global group ids [group0, group0 + ngroups)
    int32_t outer_reg;       // outer register receiving the sum
    int32_t nvar_leaves;     // IVAR instructions in the template
    int32_t node0;           // first node of its group tree in a parent's node array
    int32_t nnodes;          // nodes of the group tree (all levels)
};

struct GbGroup {
    int32_t t0, count;       // term ordinals [t0, t0 + count) of its ISUM
    int32_t bmin, bmax;      // touched blocks (-1, -1 if the template has no IVAR)
};

// ---- per-parent term tables ------------------------------------------------
// A child of a box differs from it only in the pieces of the split
// coordinates [c0, c0 + dd).  A term that touches w of them takes at most
// m^w values over all the children, so per parent the value, the midpoint
// value and the leaf adjoints of every dirty term are tabulated once per
// digit combination, and a child assembles its sums from the tables.
// Layouts depend only on the split position (c0, dd), fixed at creation.
struct GbSplitPos {
    int32_t c0, dd, block;
    int32_t dterm0, ndterm;   // dirty terms [dterm0, dterm0 + ndterm)
    int32_t tab_entries;      // combinations over all dirty terms (table rows)
    int32_t jk0;              // (coordinate of the block, sum) ranges start
    int32_t drows;            // rows of the per-parent partial tables
    int32_t seg0, nseg;       // segments [seg0, seg0 + nseg) of the dirty groups' term trees
    int32_t srows;            // rows of the per-parent segment tables
    int32_t pad;
};
// A segment of a dirty group's term tree: the aligned block of 2^level terms
// starting at dirty term dterm (relative to the split position's dterm0),
// whose in-place pairwise sum depends only on the child's digit bits
// [shift, shift + bits) (bits <= GB_TAB_SBITS).  level 0: a single term,
// read from its term row `base`; level >= 1: tabulated per parent at segment
// row base + ((r >> shift) & mask).  A group's segments cover its terms in
// order, so pushing each segment's value into the binary counter at its
// level gives the group's pairwise tree.
#define GB_TAB_SBITS 10
#define GB_TAB_SCOST 14   // a segment's table costs 2^(bits + level) additions per parent: at most 2^14
struct GbSeg {
    int32_t base;
    int32_t dterm;
    int16_t shift;
    uint16_t mask;
    int8_t sum, level;
    int16_t group;
};
struct GbDTerm {
    int16_t sum, w;           // sum index, number of split coordinates touched
    int16_t dshift, group;    // bit shift of its first digit in the child index, local group
    int32_t term;             // term ordinal within the sum
    int32_t row;              // first table row of the term (m^w rows)
};
// A leaf adjoint feeding one coordinate: dirty term, leaf, and its table
// address (row * max_leaves + leaf; the child's digits select
// base + ((r >> dshift) & mask) * max_leaves).
struct GbContrib {
    int32_t dterm, leaf;
    int32_t base;
    int16_t dshift;
    uint16_t mask;
};
// Per (coordinate of the block, sum): the sum over its contributions of the
// leaf adjoints depends only on the child's digit bits [shift, shift + bits)
// (bits <= GB_TAB_DBITS); such sums are tabulated per parent at rows
// base + ((r >> shift) & mask).  shift < 0: not tabulated.
#define GB_TAB_DBITS 6
struct GbJkD {
    int32_t base;
    int16_t shift;
    uint16_t mask;
};

// Outer VAR leaf: register and coordinate (for the gradient).
struct GbVarLeaf { int32_t reg, coord; };

// Program passed by value to kernels (pointers are device memory).
struct GbProg {
    int32_t n, B, nb;
    int32_t n_sum, n_groups;         // ISUM nodes, total groups
    int32_t n_outer, outer_root;     // outer instructions (register = index)
    int32_t n_var_leaves;
    const GbIns* outer;              // [n_outer]
    const GbIns* tins;               // all template instructions
    const GbSum* sums;               // [n_sum]
    const GbGroup* groups;           // [n_groups]
    const int2* dirty;               // [nb * n_sum]: dirty local group range per block
    const GbVarLeaf* var_leaves;     // [n_var_leaves]
    const double* const* tab64;      // [n_tables] table pointers
    const float2* const* tab32;      // [n_tables] outward float pairs (lo, hi)
    const double* l;                 // [n]
    const double* u;                 // [n]
    // block records (pool mode 2): group -> (owner block, index in its record)
    int32_t GPB, span, nrec;         // groups per record, max block span of a group, records per child
    const int2* gown;                // [n_groups]
    const int32_t* owned;            // [nb * GPB] global groups owned by each block (-1: none)
    // per-parent term tables (null when not built)
    int32_t tab_ok, m, mshift, max_rows, max_leaves, tree_nodes, max_dterm;
    const int32_t* sp_of_cyc;        // [n] split position of a cycling position (-1: unreachable)
    const GbSplitPos* sps;
    const GbDTerm* dterms;
    const int2* jk;                  // [(c1 - c0) * n_sum] per split position: contribution ranges
    const GbContrib* contribs;
    const GbJkD* jkd;                // parallel to jk: partial-table rows
    int32_t max_drows;
    const GbSeg* segs;               // term-tree segments of every split position
    int32_t max_srows, max_nseg;
    int32_t outer_sum;               // 1: the outer expression is one sum (F = that sum, adjoint [1, 1])
    int32_t outer_unit;              // 1: every sum's outer adjoint is exactly [1, 1] and no outer VAR
                                     //    leaf: the first-order test needs no reverse sweep of the outer
    int32_t samples;                 // GUB samples per box (0: midpoint; S: diagonal points j / (S + 1))
    int32_t mono_all;                // first-order test on every coordinate
    int32_t any_prod;                // some reduction is an IPROD
};

// Host-side compiled program (arrays in host memory before upload).
#ifdef __cplusplus
#include <string>
#include <vector>
struct GbHostProg {
    int32_t n = 0, B = 0, nb = 0;
    int32_t outer_root = 0;
    int32_t any_prod = 0;
    std::vector<GbIns> outer, tins;
    std::vector<GbSum> sums;
    std::vector<GbGroup> groups;
    std::vector<int2> dirty;
    std::vector<GbVarLeaf> var_leaves;
    int64_t ops_eval = 0, ops_mid = 0;   // static directed-op counts (see gb_compile.cpp)
    // block records: group ownership (a group lives in the record of its lowest touched block)
    int32_t GPB = 1, span = 0;
    std::vector<int2> gown;
    std::vector<int32_t> owned;
    // per-parent term tables
    int32_t tab_ok = 0, m = 2, mshift = 1, max_rows = 0, max_leaves = 0, tree_nodes = 0, max_dterm = 0;
    std::vector<int32_t> sp_of_cyc;
    std::vector<GbSplitPos> sps;
    std::vector<GbDTerm> dterms;
    std::vector<int2> jk;
    std::vector<GbContrib> contribs;
    std::vector<GbJkD> jkd;
    int32_t max_drows = 0;
    std::vector<GbSeg> segs;
    int32_t max_srows = 0, max_nseg = 0;
};
// Builds the per-split-position table layouts for pieces m and split width d;
// leaves tab_ok = 0 when a layout exceeds the table limits.
// sbits: largest digit-bit count of a tabulated term-tree segment (<= GB_TAB_SBITS).
void gb_build_tables(GbHostProg* P, int m, int d, int sbits = GB_TAB_SBITS);
// Compiles and validates a DAG; returns an empty string or an error message.
std::string gb_compile(const gb_node* nodes, int32_t nn, int32_t root, const int64_t* tlen,
                       int32_t ntab, int32_t n, int32_t B, GbHostProg* out);
#endif

// Order-preserving map of doubles to unsigned keys (for min reductions and
// the best-first selection).
GB_HD inline unsigned long long gb_order_key(double x) {
    union { double d; unsigned long long u; } v;
    v.d = x;
    return (v.u >> 63) ? ~v.u : (v.u | 0x8000000000000000ull);
}
GB_HD inline double gb_key_value(unsigned long long k) {
    union { double d; unsigned long long u; } v;
    v.u = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return v.d;
}

// Device-side solver state of one problem (one copy in device memory; the
// host reads it back once per generation).
struct GbState {
    long long pool;             // entries in the current pool
    long long nfree;            // slots on the free list
    long long bump;             // next never-used slot
    long long cap;              // slot capacity
    long long active;           // active entries (F_lo < RU(GUB - tol_f), not final)
    long long parents;          // parents selected this generation
    long long drops;            // entries removed by the cut-off this generation
    long long kept_old;         // entries carried over
    long long children;         // children evaluated
    long long kept32;           // children passing the FP32 pass
    long long kept;             // children inserted
    long long gen;              // generations completed
    long long sel_below;        // selection: active entries with key < sel_T
    long long sel_need;         // ties (key == sel_T) to take, the last ones in pool order
    long long sel_ties;         // active entries with key == sel_T
    long long radix_rank;       // radix select: remaining rank
    long long n32;              // length of the FP32-survivor list
    long long nfree_base;       // free-list size when the pool partition starts (set by k_stats)
    unsigned long long gub_key;     // incumbent upper bound (order key)
    unsigned long long gub_new_key; // min over this generation's samples
    unsigned long long sel_T;       // selection threshold key (~0: take all active)
    unsigned long long radix_prefix;
    unsigned long long glb_key;     // min lower bound over the pool (final pass)
    int overflow;               // survivors do not fit: generation abandoned
    int error;                  // device-side error code (bit flags)
    int halt;                   // set at the start of a generation that must not run
    int sel_mode;               // selection: 0 all active, 1 minimum key (K = 1), 2 radix select
    long long nch;              // children of this generation (parents * fan-out)
    long long rec_nfree, rec_bump;     // block records: free list size, next never-used record
    long long rec_gc;                  // block records: collections run
    int gc;                            // block records: collect before this generation's inserts
    unsigned stats_done;               // blocks of k_stats finished (the last one starts the generation)
    unsigned cc_done;                  // blocks of the child kernel finished (the last one lists the survivors)
    unsigned part_done;                // blocks of the partition finished (the last one combines their keys)
    unsigned long long min_key;        // smallest active key (K = 1 selection)
    long long evals32, evals64, mids;  // running counters
    unsigned long long ops64, ops32;   // directed-rounding operations executed by the eval kernels
    long long sel_pos;                 // K = 1: pool position of the selected entry (last with the smallest key)
    long long active_acc;              // k_stats: active entries counted so far by its blocks
    unsigned long long part_epoch;     // pool partitions started in this solve (their tile flags carry it)
    unsigned long long part_ticket;    // pool partition: next tile to hand out
};
