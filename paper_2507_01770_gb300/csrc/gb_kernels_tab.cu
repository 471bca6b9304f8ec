// Child evaluation from per-parent term tables.
//
// The paper computes each child's bounds from its parent and its index
// (Eqs. 7-11, the SPSD style of section 3.2).  Carried one step further: a
// term that touches w of the split coordinates takes at most m^w values over
// all children of a parent, so k_ptab tabulates, once per parent, the value,
// the midpoint value and the leaf adjoints of every dirty term for each digit
// combination, together with the group-sum trees of the parent's cached sums.
// A child then reads its terms from the tables, rebuilds only the path of the
// group tree above its dirty groups, and runs the outer expression and the
// first-order test.  Every value is computed by the same operations in the
// same order as the interpreter kernels, so the results are bit-identical.
#include <cuda_runtime.h>

#include "gb_child.cuh"

using namespace gb;

// Resident blocks of 128 threads per SM the one-child-per-thread kernels are
// compiled for (register budget 65536 / (128 * GB_TAB_MINB) per thread).
#ifndef GB_TAB_MINB
#define GB_TAB_MINB 7
#endif
// The same for the register-resident single-sum kernel (80 registers, no
// local memory to speak of; measured on the n = 100 chain, 4^10 children a
// launch: 27.1 ms per solve at 6 blocks, 27.7 at 5 and at 7).
#ifndef GB_TAB_MINB_REG
#define GB_TAB_MINB_REG 6
#endif
// Blocks per SM of their grid (each thread loops over children).
#ifndef GB_TAB_GRID
#define GB_TAB_GRID 32
#endif

namespace {

template <typename T> struct TabPrec;
template <> struct TabPrec<double> {
    typedef iv64 I;
    typedef double2 P2;
    static __device__ __forceinline__ I tv(const GbTabs& T, size_t i) { double2 v = T.tv64[i]; return I{v.x, v.y}; }
    static __device__ __forceinline__ I tl(const GbTabs& T, size_t i) { double2 v = T.tl64[i]; return I{v.x, v.y}; }
    static __device__ __forceinline__ I node(const GbTabs& T, size_t i) { double2 v = T.nf64[i]; return I{v.x, v.y}; }
};
template <> struct TabPrec<float> {
    typedef iv32 I;
    typedef float2 P2;
    static __device__ __forceinline__ I tv(const GbTabs& T, size_t i) { float2 v = T.tv32[i]; return I{v.x, v.y}; }
    static __device__ __forceinline__ I tl(const GbTabs& T, size_t i) { float2 v = T.tl32[i]; return I{v.x, v.y}; }
    static __device__ __forceinline__ I node(const GbTabs& T, size_t i) { float2 v = T.nf32[i]; return I{v.x, v.y}; }
};

__device__ __forceinline__ iv64 mid_node(const GbTabs& T, size_t i) { double2 v = T.nm64[i]; return iv64{v.x, v.y}; }

// ---------------------------------------------------------------------------
// k_ptab: per parent (blockIdx.y).  Blocks x < row_blocks: table row parts,
// PTAB_ITEMS per block (one warp) -- rows are (dirty term, digit
// combination) and each row has up to three independent parts: 0 the FP64
// value and leaf adjoints (one forward pass, then the reverse sweep), 1 the
// midpoint value, 2 the FP32 value and leaf adjoints.  A part is one serial
// chain of FP64 work (a template's interval operations, transcendentals
// included).  On GB300 a dependent FP64 operation takes ~30 ns and a warp's
// FP64 instruction holds the SM's FP64 pipe for ~16 clocks whatever its
// active lanes, so each part gets a warp of its own (parts in one warp would
// diverge and run one after the other), spread over the SMs.  The warp's
// lanes first stage the template's instructions and its coordinate and
// coefficient values in shared memory (all loads in flight at once), then
// lanes 0 and 1 interpret it together: both run every operation, and exp,
// sin and cos evaluate their two endpoints one per lane (itrig_pair).
// Blocks x >= row_blocks: one group tree of the parent's cached sums each
// (sum k, kind: F, midpoint, FP32), level by level.
constexpr int PTAB_T = 128;
constexpr int PTAB_ITEMS = 4;        // row parts per block: one per warp, in its lane 0
constexpr int PTAB_SMEM_DT = 256;   // dirty terms staged in shared memory for the row lookup

__host__ __device__ __forceinline__ int ptab_parts(const GbPool& pool) { return pool.fp32 ? 3 : 2; }

// One level-major pairwise group tree: the level-0 nodes (the parent's
// cached group sums) are in a[0, ngroups); every level is formed from the one
// below it.  `a` is shared memory when the tree fits (one memory round trip
// for the whole tree), else the output itself.
template <typename I, typename P2>
__device__ __forceinline__ void build_tree(P2* a, int ngroups, int& tops) {
    int off = 0;
    for (int mL = ngroups; mL > 1; mL = (mL + 1) / 2) {
        const int mN = (mL + 1) / 2;
        for (int q = threadIdx.x; q < mN; q += blockDim.x) {
            const P2 x = a[off + 2 * q];
            I v = mk<decltype(x.x)>(x.x, x.y);
            if (2 * q + 1 < mL) {
                const P2 y = a[off + 2 * q + 1];
                v = iadd(v, mk<decltype(y.x)>(y.x, y.y));
                tops += 2;
            }
            P2 o;
            o.x = v.lo;
            o.y = v.hi;
            a[off + mL + q] = o;
        }
        __syncthreads();
        off += mL;
    }
}

template <typename I, typename P2, typename C>
__device__ __forceinline__ void tree_job(const GbSum& S, const C& cache, P2* out, P2* sm, bool in_smem, int& tops) {
    P2* a = in_smem ? sm : out;
    for (int g = threadIdx.x; g < S.ngroups; g += blockDim.x) a[g] = cache[S.group0 + g];
    __syncthreads();
    build_tree<I>(a, S.ngroups, tops);
    if (in_smem)
        for (int i = threadIdx.x; i < S.nnodes; i += blockDim.x) out[i] = sm[i];
}

// The split of parent p (Eqs. 10-11 with the rounding reading: boundary t of
// [lo, hi] is RN(lo + RN(RN(RN(hi - lo) / m) * t)), boundary 0 = lo, boundary
// m = hi; the division by m = 2 or 4 is the exact product by 1 / m): its
// split position (first coordinate, coordinates split, block, next cycling
// position) and the m + 1 boundaries of each split coordinate with their
// outward floats, computed by threads 0 .. dmax-1 into the block's shared
// memory (and, when `publish`, into the parent buffers for the later kernels).
__device__ __forceinline__ int4 parent_split(const GbProg& P, const GbPool& pool, const GbParents& par,
                                             const GbSplit& sp, long long p, unsigned slot, int cyc, double* bnd,
                                             float* brd, float* bru, bool publish) {
    const int n = P.n, B = P.B;
    const int c = cyc & 0x7fffffff, b = c / B, e = min((b + 1) * B, n);
    const int dd = min(sp.d, e - c), nxt = (c + dd == n) ? 0 : c + dd;
    const int4 info = make_int4(c, dd, b, nxt);
    const int k = threadIdx.x, ms = sp.m + 1;
    if (k < dd) {
        const iv64 pj = box_view64(pool, slot).get(c + k);
        const double lo = pj.lo, hi = pj.hi;
        const double q = __dmul_rn(__dsub_rn(hi, lo), sp.m == 2 ? 0.5 : 0.25);
        for (int t = 0; t <= sp.m; t++) {
            const double v = (t == 0) ? lo : (t == sp.m ? hi : __dadd_rn(lo, __dmul_rn(q, (double)t)));
            bnd[k * ms + t] = v;
            brd[k * ms + t] = __double2float_rd(v);
            bru[k * ms + t] = __double2float_ru(v);
            if (publish) {
                const size_t o = ((size_t)p * sp.dmax + k) * ms + t;
                par.bnd[o] = v;
                par.bnd_rd[o] = __double2float_rd(v);
                par.bnd_ru[o] = __double2float_ru(v);
            }
        }
    }
    if (publish && k == 0) par.info[p] = info;
    return info;
}

__global__ void __launch_bounds__(PTAB_T) k_ptab(GbProg P, GbPool pool, GbParents par, GbTabs T, GbSplit sp,
                                                 int row_blocks, GbState* st, GbEntries E, int from_sel) {
    gb_grid_trigger();
    gb_grid_wait();
    if (st->halt) return;
    extern __shared__ double2 s_tree[];   // T.max_sum_nodes entries when the trees fit
    __shared__ double s_bnd[GB_MAX_SPLIT_D * 5];
    __shared__ float s_brd[GB_MAX_SPLIT_D * 5], s_bru[GB_MAX_SPLIT_D * 5];
    const long long p = blockIdx.y;
    // from_sel: the one parent is pool entry sel_pos (the partition, which
    // writes the parent count, may be running)
    if (!from_sel && p >= st->parents) return;
    const long long q = from_sel ? st->sel_pos : 0;
    const unsigned slot = from_sel ? E.slot[q] : par.slot[p];
    const int cyc = from_sel ? E.cyc[q] : par.cyc[p];
    if (blockIdx.x == 0 && p == 0 && threadIdx.x == 0) {   // the generation's counters (k_prep's part)
        if (from_sel) {
            par.slot[0] = slot;
            par.cyc[0] = cyc;
            par.flo[0] = E.flo[q];
        }
        st->gub_new_key = st->gub_key;
        st->kept = 0;
        st->kept32 = 0;
        st->n32 = 0;
        st->children = 0;
        st->overflow = 0;
    }
    // the split position's tables (they depend on the cycling position only:
    // its dirty terms are staged while the split's box loads are in flight)
    const int spi = P.sp_of_cyc[cyc & 0x7fffffff];
    const bool rows = (int)blockIdx.x < row_blocks;
    __shared__ int s_row[PTAB_SMEM_DT];
    GbSplitPos SP{};
    bool staged = false;
    if (rows && spi >= 0) {
        SP = P.sps[spi];
        staged = SP.ndterm <= PTAB_SMEM_DT;
        if (staged)
            for (int t = threadIdx.x; t < SP.ndterm; t += blockDim.x) s_row[t] = P.dterms[SP.dterm0 + t].row;
    }
    int4 info = make_int4(0, 0, 0, 0);
    if (rows) info = parent_split(P, pool, par, sp, p, slot, cyc, s_bnd, s_brd, s_bru, blockIdx.x == 0);
    __syncthreads();
    if (spi < 0) return;
    if (!rows) {
        // group tree job (k, kind)
        const int kinds = pool.fp32 ? 3 : 2;
        const int job = blockIdx.x - row_blocks;
        if (job >= P.n_sum * kinds) return;
        const int k = job % P.n_sum, kind = job / P.n_sum;
        const GbSum S = P.sums[k];
        const size_t nb = (size_t)p * T.tree_nodes + S.node0;
        const bool in_smem = T.tree_smem != 0;
        int tops = 0;
        if (kind == 0) tree_job<iv64>(S, cache64(pool, P, slot, 0), T.nf64 + nb, s_tree, in_smem, tops);
        else if (kind == 1) tree_job<iv64>(S, cache64(pool, P, slot, 1), T.nm64 + nb, s_tree, in_smem, tops);
        else tree_job<iv32>(S, cache32(pool, P, slot), T.nf32 + nb, (float2*)s_tree, in_smem, tops);
        warp_add_ops(tops, kind == 2 ? &st->ops32 : &st->ops64);
        return;
    }
    const int parts = ptab_parts(pool);
    int ops = 0, ops32 = 0, spare = 0;   // (lane 1's interpreter counts go to `spare`)
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // per warp: the template's instructions and load values (stage_term)
    __shared__ GbIns s_ins[PTAB_ITEMS][GB_MAX_TREGS];
    __shared__ double2 s_pre[PTAB_ITEMS][GB_MAX_TREGS];
    for (int item = blockIdx.x * PTAB_ITEMS + wib; item < SP.tab_entries * parts; item += row_blocks * PTAB_ITEMS) {
        const int row = item / parts, part = item - row * parts;
        // the dirty term owning this row (rows are contiguous per term)
        int lo = 0, hi = SP.ndterm - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            const int r0 = staged ? s_row[mid] : P.dterms[SP.dterm0 + mid].row;
            if (r0 <= row) lo = mid; else hi = mid - 1;
        }
        const GbDTerm D = P.dterms[SP.dterm0 + lo];
        const unsigned r = (unsigned)(row - D.row) << D.dshift;   // a child index with these digits
        const GbSum S = P.sums[D.sum];
        const int i = S.first + D.term * S.step;
        const size_t orow = (size_t)p * T.max_rows + row;
        const GbIns* ins = s_ins[wib];
        if (part < 2) {
            iv64* pre = reinterpret_cast<iv64*>(s_pre[wib]);
            View<double> X = box_view64(pool, slot);
            X.blo = s_bnd;
            X.bhi = s_bnd;
            X.c0 = info.x;
            X.dd = info.y;
            X.mshift = sp.mshift;
            X.mstride = sp.m + 1;
            X.r = r;
            if (part == 1) {
                stage_term<double>(P, S, i, MidView{X}, s_ins[wib], pre, lane);
                if (lane < 2) {
                    iv64 R[GB_MAX_TREGS];
                    const iv64 v = term_fwd<double, MidView, true>(P, S, i, MidView{X}, R, lane ? spare : ops, ins, pre);
                    if (lane == 0) T.tm64[orow] = make_double2(v.lo, v.hi);
                }
            } else {
                stage_term<double>(P, S, i, X, s_ins[wib], pre, lane);
                if (lane < 2) {
                    int& o = lane ? spare : ops;
                    iv64 R[GB_MAX_TREGS], RA[GB_MAX_TREGS];
                    const iv64 v = term_fwd<double, View<double>, true>(P, S, i, X, R, o, ins, pre);
                    for (int t = 0; t < S.nins; t++) RA[t] = iv64{0.0, 0.0};
                    RA[S.nins - 1] = iv64{1.0, 1.0};
                    reverse_sweep<double, true>(ins, S.nins, R, RA, o);
                    if (lane == 0) {
                        T.tv64[orow] = make_double2(v.lo, v.hi);
                        int leaf = 0;
                        for (int t = 0; t < S.nins; t++) {
                            if (ins[t].op != D_IVAR) continue;
                            T.tl64[orow * T.max_leaves + leaf] = make_double2(RA[t].lo, RA[t].hi);
                            leaf++;
                        }
                    }
                }
            }
        } else {
            iv32* pre = reinterpret_cast<iv32*>(s_pre[wib]);
            View<float> X32 = box_view32(pool, slot);
            X32.blo = s_brd;
            X32.bhi = s_bru;
            X32.c0 = info.x;
            X32.dd = info.y;
            X32.mshift = sp.mshift;
            X32.mstride = sp.m + 1;
            X32.r = r;
            stage_term<float>(P, S, i, X32, s_ins[wib], pre, lane);
            if (lane < 2) {
                int& o = lane ? spare : ops32;
                iv32 R32[GB_MAX_TREGS], RA32[GB_MAX_TREGS];
                const iv32 f = term_fwd<float, View<float>, true>(P, S, i, X32, R32, o, ins, pre);
                for (int t = 0; t < S.nins; t++) RA32[t] = iv32{0.f, 0.f};
                RA32[S.nins - 1] = iv32{1.f, 1.f};
                reverse_sweep<float, true>(ins, S.nins, R32, RA32, o);
                if (lane == 0) {
                    T.tv32[orow] = make_float2(f.lo, f.hi);
                    int leaf = 0;
                    for (int t = 0; t < S.nins; t++) {
                        if (ins[t].op != D_IVAR) continue;
                        T.tl32[orow * T.max_leaves + leaf] = make_float2(RA32[t].lo, RA32[t].hi);
                        leaf++;
                    }
                }
            }
        }
        __syncwarp();   // the staging is reused by the warp's next item
    }
    warp_add_ops(ops, &st->ops64);   // one atomic per warp (every lane reaches here)
    warp_add_ops(ops32, &st->ops32);
}

// ---------------------------------------------------------------------------
// k_ptab_d: per parent (blockIdx.y), from the term rows of k_ptab (runs
// after it): (1) the partial tables: for each (coordinate of the block, sum)
// tabulated by the layout and each digit combination of its bits, the serial
// sum of the leaf adjoints of its contributions (the order tab_partial uses),
// one thread per entry; (2) the segment tables: for each term-tree segment
// of level >= 1 and each combination of its digit bits, the in-place
// pairwise sum of its 2^level terms (F, midpoint, FP32), one warp per entry.
// A segment is an aligned power-of-two block, so its pairwise tree is a
// perfect binary tree: lane i holds term i (or, above 32 terms, the pairwise
// sum of its aligned run of terms) and at level s lane i adds lane i + s --
// the left node plus the right node, as the serial tree does, in log2 steps
// instead of 2^level dependent ones.
template <typename I> __device__ __forceinline__ I shfl_down_iv(I v, int d) {
    v.lo = __shfl_down_sync(0xffffffffu, v.lo, d);
    v.hi = __shfl_down_sync(0xffffffffu, v.hi, d);
    return v;
}

__global__ void __launch_bounds__(128) k_ptab_d(GbProg P, GbPool pool, GbParents par, GbTabs T,
                                                GbState* st, int fixed) {
    gb_grid_trigger();
    gb_grid_wait();
    if (st->halt) return;
    const long long p = blockIdx.y;
    if (!fixed && p >= st->parents) return;
    const int4 info = par.info[p];
    const int spi = P.sp_of_cyc[info.x];
    if (spi < 0) return;
    const GbSplitPos SP = P.sps[spi];
    const int c0 = info.z * P.B, c1 = min(P.n, c0 + P.B);
    const int nent = (c1 - c0) * P.n_sum;
    const double2* tl = T.tl64 + (size_t)p * T.max_rows * T.max_leaves;
    const float2* tl32 = pool.fp32 ? T.tl32 + (size_t)p * T.max_rows * T.max_leaves : nullptr;
    const int nd_items = nent << GB_TAB_DBITS;
    const int lane = threadIdx.x & 31;
    int ops = 0, ops32 = 0;
    // (1) partial tables
    for (int item = blockIdx.x * blockDim.x + threadIdx.x; item < nd_items; item += gridDim.x * blockDim.x) {
        const int e = item >> GB_TAB_DBITS, c = item & ((1 << GB_TAB_DBITS) - 1);
        const GbJkD J = P.jkd[SP.jk0 + e];
        if (J.shift < 0 || c > (int)J.mask) continue;
        const int2 rg = P.jk[SP.jk0 + e];
        const unsigned r = (unsigned)c << J.shift;
        iv64 D{0.0, 0.0};
        iv32 D32{0.f, 0.f};
        for (int q = rg.x; q < rg.y; q++) {
            const GbContrib C = P.contribs[q];
            const int at = C.base + (int)((r >> C.dshift) & C.mask) * T.max_leaves;
            const double2 v = tl[at];
            D = q > rg.x ? iadd(D, iv64{v.x, v.y}) : iv64{v.x, v.y};
            if (tl32) {
                const float2 v32 = tl32[at];
                D32 = q > rg.x ? iadd(D32, iv32{v32.x, v32.y}) : iv32{v32.x, v32.y};
            }
        }
        if (rg.y - rg.x > 1) {
            ops += 2 * (rg.y - rg.x - 1);
            if (tl32) ops32 += 2 * (rg.y - rg.x - 1);
        }
        const size_t o = (size_t)p * T.max_drows + J.base + c;
        T.td64[o] = make_double2(D.lo, D.hi);
        if (tl32) T.td32[o] = make_float2(D32.lo, D32.hi);
    }
    // (2) segment tables
    const int nw_items = SP.nseg << GB_TAB_SBITS;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const size_t rb = (size_t)p * T.max_rows;
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nw_items; w += nwarps) {
        const int si = w >> GB_TAB_SBITS, c = w & ((1 << GB_TAB_SBITS) - 1);
        const GbSeg G = P.segs[SP.seg0 + si];
        if (G.level == 0 || c > (int)G.mask) continue;   // the same for the whole warp
        const unsigned r = (unsigned)c << G.shift;
        const int L = G.level, sub = L > 5 ? L - 5 : 0, width = 1 << (L - sub);
        iv64 f{0.0, 0.0}, m{0.0, 0.0};
        iv32 f32{0.f, 0.f};
        if (lane < width) {
            Tree<iv64> tf, tm;
            Tree<iv32> t32;
            tf.init();
            tm.init();
            t32.init();
            for (int t = lane << sub; t < (lane + 1) << sub; t++) {
                const GbDTerm D = P.dterms[SP.dterm0 + G.dterm + t];
                const size_t at = rb + D.row + ((r >> D.dshift) & ((1u << (D.w * P.mshift)) - 1u));
                const double2 a = T.tv64[at], b = T.tm64[at];
                tf.push(iv64{a.x, a.y});
                tm.push(iv64{b.x, b.y});
                if (tl32) {
                    const float2 x = T.tv32[at];
                    t32.push(iv32{x.x, x.y});
                }
            }
            f = tf.result();
            m = tm.result();
            if (tl32) f32 = t32.result();
        }
        for (int d = 1; d < width; d <<= 1) {
            const iv64 of = shfl_down_iv(f, d), om = shfl_down_iv(m, d);
            const iv32 o32 = shfl_down_iv(f32, d);
            if ((lane & (2 * d - 1)) == 0) {
                f = iadd(f, of);
                m = iadd(m, om);
                if (tl32) f32 = iadd(f32, o32);
            }
        }
        if (lane == 0) {
            ops += 4 * ((1 << L) - 1);   // F and midpoint trees
            if (tl32) ops32 += 2 * ((1 << L) - 1);
            const size_t o = (size_t)p * T.max_srows + G.base + c;
            T.ts64[o] = make_double2(f.lo, f.hi);
            T.tsm64[o] = make_double2(m.lo, m.hi);
            if (tl32) T.ts32[o] = make_float2(f32.lo, f32.hi);
        }
    }
    warp_add_ops(ops, &st->ops64);   // one atomic per warp (every lane reaches here)
    warp_add_ops(ops32, &st->ops32);
}

// ---------------------------------------------------------------------------
// Path of sum k's pairwise group tree above its dirty groups [dr.x, dr.y)
// (values cur[0 .. dr.y - dr.x)), with the parent's tree nodes (node(i),
// level-major) for the clean siblings; returns the sum.
template <typename I, typename N>
__device__ __forceinline__ I tab_path(const GbSum& S, int2 dr, I* cur, N node, int& ops) {
    I tmp[GB_TAB_MAX_DIRTY];
    if (S.ngroups == 0 || S.nnodes <= 0) {
        I z;
        z.lo = 0;
        z.hi = 0;
        return z;
    }
    int lo = dr.x, hi = dr.y, off = 0;
    if (lo >= hi) return node(S.nnodes - 1);   // no dirty group: the parent's root
    for (int mL = S.ngroups; mL > 1; mL = (mL + 1) / 2) {
        const int nlo = lo >> 1, nhi = ((hi - 1) >> 1) + 1;
        for (int q = nlo; q < nhi; q++) {
            const int a = 2 * q;
            I left = (a >= lo && a < hi) ? cur[a - lo] : node(off + a);
            I v = left;
            if (a + 1 < mL) {
                I right = (a + 1 >= lo && a + 1 < hi) ? cur[a + 1 - lo] : node(off + a + 1);
                v = iadd(left, right);
                ops += 2;
            }
            tmp[q - nlo] = v;
        }
        for (int q = 0; q < nhi - nlo; q++) cur[q] = tmp[q];
        lo = nlo;
        hi = nhi;
        off += mL;
    }
    return cur[0];
}

// tab_path for a warp whose lanes all walk the same path (one child per
// warp): the clean sibling nodes the walk reads depend only on the tree's
// shape and the dirty range, so they are listed first (lane t takes the t-th
// one the walk will read) and loaded by all lanes at once, one round of
// memory latency instead of one per level; the walk then takes each from its
// lane.  Same operations in the same order as tab_path, so the same sum,
// returned in lane 0 (cur is read in lane 0 only).
template <typename I, typename N>
__device__ __forceinline__ I tab_path_w(const GbSum& S, int2 dr, I* cur, N node, int lane, int& ops) {
    if (S.ngroups == 0 || S.nnodes <= 0) {
        I z;
        z.lo = 0;
        z.hi = 0;
        return z;
    }
    if (dr.x >= dr.y) return node(S.nnodes - 1);   // no dirty group: the parent's root
    int mine = -1, cnt = 0;
    {
        int lo = dr.x, hi = dr.y, off = 0;
        for (int mL = S.ngroups; mL > 1; mL = (mL + 1) / 2) {
            const int nlo = lo >> 1, nhi = ((hi - 1) >> 1) + 1;
            for (int q = nlo; q < nhi; q++) {
                const int a = 2 * q;
                if (!(a >= lo && a < hi)) mine = cnt++ == lane ? off + a : mine;
                if (a + 1 < mL && !(a + 1 >= lo && a + 1 < hi)) mine = cnt++ == lane ? off + a + 1 : mine;
            }
            lo = nlo;
            hi = nhi;
            off += mL;
        }
    }
    I pre;
    pre.lo = 0;
    pre.hi = 0;
    if (mine >= 0) pre = node(mine);
    I tmp[GB_TAB_MAX_DIRTY];
    int lo = dr.x, hi = dr.y, off = 0, used = 0;
    // every lane follows the walk (the shuffles), lane 0 alone computes it:
    // cur and tmp are touched by one thread per warp
    auto take = [&](int idx) {
        const I v = shfl_iv(pre, used & 31);
        return used++ < 32 ? v : node(idx);
    };
    for (int mL = S.ngroups; mL > 1; mL = (mL + 1) / 2) {
        const int nlo = lo >> 1, nhi = ((hi - 1) >> 1) + 1;
        for (int q = nlo; q < nhi; q++) {
            const int a = 2 * q;
            const bool la = a >= lo && a < hi, lb = a + 1 >= lo && a + 1 < hi;
            I left = la ? pre : take(off + a);
            I right = left;
            if (a + 1 < mL) right = lb ? pre : take(off + a + 1);
            if (lane == 0) {
                if (la) left = cur[a - lo];
                I v = left;
                if (a + 1 < mL) {
                    if (lb) right = cur[a + 1 - lo];
                    v = iadd(left, right);
                }
                tmp[q - nlo] = v;
            }
            if (a + 1 < mL) ops += 2;
        }
        if (lane == 0)
            for (int q = 0; q < nhi - nlo; q++) cur[q] = tmp[q];
        lo = nlo;
        hi = nhi;
        off += mL;
    }
    return cur[0];   // defined in lane 0
}

// tab_path for 32 lanes that walk the same path (same tree and dirty range)
// over their own dirty values: the sibling nodes are loaded once across the
// lanes (lane t the t-th one the walk reads) and handed out by shuffles;
// every lane computes its own walk.  Same operations in the same order as
// tab_path.
template <typename I, typename N>
__device__ __forceinline__ I tab_path_lanes(const GbSum& S, int2 dr, I* cur, N node, int lane, int& ops) {
    if (S.ngroups == 0 || S.nnodes <= 0) {
        I z;
        z.lo = 0;
        z.hi = 0;
        return z;
    }
    if (dr.x >= dr.y) return node(S.nnodes - 1);
    int mine = -1, cnt = 0;
    {
        int lo = dr.x, hi = dr.y, off = 0;
        for (int mL = S.ngroups; mL > 1; mL = (mL + 1) / 2) {
            const int nlo = lo >> 1, nhi = ((hi - 1) >> 1) + 1;
            for (int q = nlo; q < nhi; q++) {
                const int a = 2 * q;
                if (!(a >= lo && a < hi)) mine = cnt++ == lane ? off + a : mine;
                if (a + 1 < mL && !(a + 1 >= lo && a + 1 < hi)) mine = cnt++ == lane ? off + a + 1 : mine;
            }
            lo = nlo;
            hi = nhi;
            off += mL;
        }
    }
    I pre;
    pre.lo = 0;
    pre.hi = 0;
    if (mine >= 0) pre = node(mine);
    I tmp[GB_TAB_MAX_DIRTY];
    int lo = dr.x, hi = dr.y, off = 0, used = 0;
    auto take = [&](int idx) {
        const I v = shfl_iv(pre, used & 31);
        return used++ < 32 ? v : node(idx);
    };
    for (int mL = S.ngroups; mL > 1; mL = (mL + 1) / 2) {
        const int nlo = lo >> 1, nhi = ((hi - 1) >> 1) + 1;
        for (int q = nlo; q < nhi; q++) {
            const int a = 2 * q;
            const bool la = a >= lo && a < hi, lb = a + 1 >= lo && a + 1 < hi;
            I left = la ? cur[a - lo] : take(off + a);
            I v = left;
            if (a + 1 < mL) {
                const I right = lb ? cur[a + 1 - lo] : take(off + a + 1);
                v = iadd(left, right);
                ops += 2;
            }
            tmp[q - nlo] = v;
        }
        for (int q = 0; q < nhi - nlo; q++) cur[q] = tmp[q];
        lo = nlo;
        hi = nhi;
        off += mL;
    }
    return cur[0];
}

// ---------------------------------------------------------------------------
// k_child_sums (one child per warp): every child's sums before the child
// kernel, one thread per (child, sum, kind) -- kind 0 F, 1 midpoint, 2 FP32.
// A thread takes its sum's dirty groups from the term-tree segments (the
// binary counter over the segments in order) and the path of the group tree
// above them (tab_path), the same operations in the same order as the child
// kernels' own assembly, so the same values; it stores the dirty group
// values too, for the materialisation of the survivors.  Consecutive threads
// are consecutive children of the same (sum, kind), so a warp follows one
// control path; the ~10^4 short chains run side by side instead of one
// child's chains one after another in a warp.
template <typename I, typename P2>
__device__ __forceinline__ void child_sum(const GbProg& P, const GbSplitPos& SP, int k, int blk, unsigned r,
                                          const P2* trow, const P2* tseg, const P2* nodes, I* gout, I* sout,
                                          bool lanes, int& ops) {
    const GbSum S = P.sums[k];
    const int2 dr = P.dirty[blk * P.n_sum + k];
    int sg = SP.seg0;
    const int send = SP.seg0 + SP.nseg;
    while (sg < send) {   // the run of (k, first dirty group): segments are ordered by sum, group, term
        const GbSeg G = P.segs[sg];
        if (G.sum > k || (G.sum == k && G.group >= dr.x)) break;
        sg++;
    }
    I cur[GB_TAB_MAX_DIRTY];
    for (int g = dr.x; g < dr.y; g++) {
        Tree<I> tr;
        tr.init();
        int ns = 0;
        while (sg < send) {
            const GbSeg G = P.segs[sg];
            if (G.sum != k || G.group != g) break;
            const int at = G.base + (int)((r >> G.shift) & G.mask);
            const P2 v = G.level ? tseg[at] : trow[at];
            tr.push_level(mk<decltype(v.x)>(v.x, v.y), G.level);
            ns++;
            sg++;
        }
        ops += 2 * (ns > 0 ? ns - 1 : 0);
        cur[g - dr.x] = tr.result();
        gout[k * GB_TAB_MAX_DIRTY + (g - dr.x)] = cur[g - dr.x];
    }
    auto node = [&](int i) { const P2 v = nodes[S.node0 + i]; return mk<decltype(v.x)>(v.x, v.y); };
    *sout = lanes ? tab_path_lanes(S, dr, cur, node, threadIdx.x & 31, ops) : tab_path(S, dr, cur, node, ops);
}

// The first-order verdict of one (parent, kind, block coordinate, digit
// combination): defined after tab_partial and mono_hit below.
__device__ void mono_fill(const GbProg& P, const GbPool& pool, const GbParents& par, const GbTabs& Tb,
                          const GbSplit& sp, long long u, long long npar, int& ops64, int& ops32);

__global__ void __launch_bounds__(128) k_child_sums(GbProg P, GbPool pool, GbParents par, GbTabs Tb, GbSplit sp,
                                                    long long Cmax, int kinds, GbState* st, long long nch_fixed,
                                                    long long mv_base) {
    gb_grid_trigger();
    gb_grid_wait();
    if (st->halt) return;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= mv_base) {   // whole blocks past the child sums: the verdict tables
        int o64 = 0, o32 = 0;
        const long long nch = nch_fixed >= 0 ? nch_fixed : st->nch;
        mono_fill(P, pool, par, Tb, sp, t - mv_base, nch >> sp.flog2, o64, o32);
        warp_add_ops(o64, &st->ops64);
        warp_add_ops(o32, &st->ops32);
        return;
    }
    const long long ci = t % Cmax, rest = t / Cmax;
    const int k = (int)(rest % (P.n_sum > 0 ? P.n_sum : 1)), kind = (int)(rest / (P.n_sum > 0 ? P.n_sum : 1));
    int ops = 0;
    // the warp's 32 children share one path when they share a parent and a
    // (sum, kind) and all of them are evaluated (the decision is the warp's)
    const long long t0 = t - (threadIdx.x & 31);
    bool lanes = t0 % Cmax + 31 < Cmax && (t0 % Cmax) >> sp.flog2 == (t0 % Cmax + 31) >> sp.flog2 &&
                 t0 + 31 < (long long)gridDim.x * blockDim.x;
    const bool live0 = P.n_sum > 0 && kind < kinds && ci < (nch_fixed >= 0 ? nch_fixed : st->nch);
    ChildCtx c{};
    int spi = -1;
    if (live0) {
        c = child_ctx(par, ci, sp);
        spi = c.valid ? P.sp_of_cyc[c.info.x] : -1;
    }
    if (lanes) lanes = __all_sync(0xffffffffu, live0 && spi >= 0);
    {
        if (live0 && spi >= 0) {
            const GbSplitPos SP = P.sps[spi];
            const size_t rowb = (size_t)c.p * Tb.max_rows, segb = (size_t)c.p * Tb.max_srows,
                         nodeb = (size_t)c.p * Tb.tree_nodes;
            const size_t so = (size_t)ci * P.n_sum + k, go = (size_t)ci * GB_CG;
            if (kind == 0)
                child_sum<iv64>(P, SP, k, c.info.z, c.r, Tb.tv64 + rowb, Tb.ts64 + segb, Tb.nf64 + nodeb,
                                (iv64*)(Tb.cg64 + go), (iv64*)(Tb.cs64 + so), lanes, ops);
            else if (kind == 1)
                child_sum<iv64>(P, SP, k, c.info.z, c.r, Tb.tm64 + rowb, Tb.tsm64 + segb, Tb.nm64 + nodeb,
                                (iv64*)(Tb.cgm64 + go), (iv64*)(Tb.csm64 + so), lanes, ops);
            else
                child_sum<iv32>(P, SP, k, c.info.z, c.r, Tb.tv32 + rowb, Tb.ts32 + segb, Tb.nf32 + nodeb,
                                (iv32*)(Tb.cg32 + go), (iv32*)(Tb.cs32 + so), lanes, ops);
        }
    }
    warp_add_ops(kind < 2 ? ops : 0, &st->ops64);
    warp_add_ops(kind == 2 ? ops : 0, &st->ops32);
}

// Sum k of a child (FP32 tables): dirty group values from the term-tree
// segments, then the path of the pairwise group tree above them with the
// parent's nodes for the clean siblings.
__device__ __forceinline__ iv32 tab_sum32(const GbProg& P, const GbTabs& Tb, long long p, const GbSplitPos& SP,
                                          int k, int blk, unsigned r, int& sg, int& ops) {
    const GbSum S = P.sums[k];
    const int2 dr = P.dirty[blk * P.n_sum + k];
    const float2* tv = Tb.tv32 + (size_t)p * Tb.max_rows;
    const float2* ts = Tb.ts32 + (size_t)p * Tb.max_srows;
    const float2* nfk = Tb.nf32 + (size_t)p * Tb.tree_nodes + S.node0;
    const int send = SP.seg0 + SP.nseg;
    iv32 cur[GB_TAB_MAX_DIRTY];
    for (int g = dr.x; g < dr.y; g++) {
        Tree<iv32> tr;
        tr.init();
        int ns = 0;
        while (sg < send) {
            const GbSeg G = P.segs[sg];
            if (G.sum != k || G.group != g) break;
            const int at = G.base + (int)((r >> G.shift) & G.mask);
            const float2 v = G.level ? ts[at] : tv[at];
            tr.push_level(iv32{v.x, v.y}, G.level);
            ns++;
            sg++;
        }
        ops += 2 * (ns > 0 ? ns - 1 : 0);
        cur[g - dr.x] = tr.result();
    }
    return tab_path(S, dr, cur, [&](int i) { const float2 v = nfk[i]; return iv32{v.x, v.y}; }, ops);
}

// First-order test from the tables (same accumulation order as block_mono).
template <typename T>
__device__ __forceinline__ const typename TabPrec<T>::P2* leaf_tab(const GbTabs& Tb, long long p);
template <>
__device__ __forceinline__ const double2* leaf_tab<double>(const GbTabs& Tb, long long p) {
    return Tb.tl64 + (size_t)p * Tb.max_rows * Tb.max_leaves;
}
template <>
__device__ __forceinline__ const float2* leaf_tab<float>(const GbTabs& Tb, long long p) {
    return Tb.tl32 + (size_t)p * Tb.max_rows * Tb.max_leaves;
}

template <typename T>
__device__ __forceinline__ const typename TabPrec<T>::P2* part_tab(const GbTabs& Tb, long long p);
template <>
__device__ __forceinline__ const double2* part_tab<double>(const GbTabs& Tb, long long p) {
    return Tb.td64 + (size_t)p * Tb.max_drows;
}
template <>
__device__ __forceinline__ const float2* part_tab<float>(const GbTabs& Tb, long long p) {
    return Tb.td32 + (size_t)p * Tb.max_drows;
}

// Value of the outer expression (F from the sums).
template <typename T, typename V>
__device__ __forceinline__ typename TabPrec<T>::I outer_value(const GbProg& P, const V& X,
                                                              const typename TabPrec<T>::I* sums,
                                                              typename TabPrec<T>::I* O, int& ops) {
    return P.outer_sum ? sums[0] : outer_fwd<T>(P, X, sums, O, ops);
}

// Interval partial of coordinate j (c0 = block start) from the outer leaves
// and the tabulated leaf adjoints; `unit` marks sums whose outer adjoint is
// exactly [1, 1] (a plain sum: the product adj * D equals D and is skipped);
// additions to an exact [0, 0] start are skipped too (they return the other
// operand's value).
template <typename T>
__device__ __forceinline__ typename TabPrec<T>::I tab_partial(const GbProg& P, const GbTabs& Tb,
                                                              const typename TabPrec<T>::P2* tl,
                                                              const typename TabPrec<T>::P2* td,
                                                              const GbSplitPos& SP, int j, int c0, unsigned r,
                                                              const typename TabPrec<T>::I* OA, unsigned unit,
                                                              int& ops) {
    typedef typename TabPrec<T>::I I;
    I g;
    bool have = false;
    for (int v = 0; v < P.n_var_leaves; v++) {
        GbVarLeaf L = P.var_leaves[v];
        if (L.coord != j) continue;
        if (have) g = iadd(g, OA[L.reg]), ops += 2;
        else g = OA[L.reg], have = true;
    }
    for (int k = 0; k < P.n_sum; k++) {
        const int at = SP.jk0 + (j - c0) * P.n_sum + k;
        const int2 rg = P.jk[at];
        if (rg.x == rg.y) continue;
        I Dk;
        const GbJkD J = P.jkd[at];
        if (J.shift >= 0) {   // tabulated per parent (k_ptab_d)
            const typename TabPrec<T>::P2 e = td[J.base + (int)((r >> J.shift) & J.mask)];
            Dk = mk<T>(e.x, e.y);
        } else {
            for (int q = rg.x; q < rg.y; q++) {
                const GbContrib C = P.contribs[q];
                const unsigned combo = (r >> C.dshift) & C.mask;
                const typename TabPrec<T>::P2 e = tl[C.base + (int)combo * Tb.max_leaves];
                const I v = mk<T>(e.x, e.y);
                if (q > rg.x) Dk = iadd(Dk, v), ops += 2;
                else Dk = v;
            }
        }
        I term;
        if ((unit >> k) & 1u) term = Dk;
        else term = imul(OA[P.sums[k].outer_reg], Dk), ops += 2;
        if (have) g = iadd(g, term), ops += 2;
        else g = term, have = true;
    }
    if (!have) g = mk<T>((T)0, (T)0);
    return g;
}

// Sums whose outer adjoint is exactly [1, 1].
template <typename I>
__device__ __forceinline__ unsigned unit_sums(const GbProg& P, const I* OA) {
    unsigned unit = 0;
    for (int k = 0; k < P.n_sum; k++) {
        const I a = OA[P.sums[k].outer_reg];
        if (is_one(a.lo) && is_one(a.hi)) unit |= 1u << k;
    }
    return unit;
}

// The first-order test discards the box when a partial has a fixed sign and
// the box does not touch the bound the sign points to.
__device__ __forceinline__ bool mono_hit(const GbProg& P, const View<double>& X64, int j, bool pos, bool neg) {
    if (!pos && !neg) return false;
    const iv64 x = X64.get(j);
    return (pos && !same_value(x.lo, __ldg(P.l + j))) || (neg && !same_value(x.hi, __ldg(P.u + j)));
}

// The digit bits of a child index that block coordinate j's first-order
// verdict depends on, when its objective has unit outer adjoints and no
// coordinate in the outer expression: the tabulated partial-table field of
// each sum with contributions to j (shift, mask) and, for a split
// coordinate, its own digit (its bounds decide the boundary condition).
// Returns false when a sum's partial is not tabulated (it is summed per
// child from its contributions) or the bits span more than GB_MV_BITS; else
// [lo, lo + nb).  `meta(k, x, y, shift, mask)` gives sum k's entry.
template <typename M>
__device__ __forceinline__ bool mv_bits(int n_sum, M meta, int jrel, int dd, int mshift, int& lo, int& nb) {
    int a = 32, b = 0;
    for (int k = 0; k < n_sum; k++) {
        int x, y, shift;
        unsigned mask;
        meta(k, x, y, shift, mask);
        if (x == y) continue;
        if (shift < 0) return false;
        if (mask == 0) continue;
        a = min(a, shift);
        b = max(b, shift + 32 - __clz(mask));
    }
    if (jrel >= 0 && jrel < dd) {
        a = min(a, jrel * mshift);
        b = max(b, (jrel + 1) * mshift);
    }
    if (b <= a) {
        lo = 0;
        nb = 0;
        return true;
    }
    if (b - a > GB_MV_BITS) return false;
    lo = a;
    nb = b - a;
    return true;
}

// Verdict table entry u (parent, kind, block coordinate, digit combination):
// the partial of the coordinate and the first-order test for a child whose
// digits are that combination (zero elsewhere: nothing else is read), with
// the operations tab_mono_w performs for every child, so its lookup gives
// the same verdict.
__device__ void mono_fill(const GbProg& P, const GbPool& pool, const GbParents& par, const GbTabs& Tb,
                          const GbSplit& sp, long long u, long long npar, int& ops64, int& ops32) {
    const int kinds = Tb.mv32 ? 2 : 1;
    const long long per_p = (long long)P.B * kinds << GB_MV_BITS;
    const long long p = u / per_p;
    const long long rem = u - p * per_p;
    const int kind = (int)(rem / ((long long)P.B << GB_MV_BITS));
    const int jl = (int)((rem >> GB_MV_BITS) % P.B), combo = (int)(rem & ((1 << GB_MV_BITS) - 1));
    if (!Tb.mv64 || p >= npar) return;
    const int4 info = par.info[p];
    const int spi = P.sp_of_cyc[info.x];
    if (spi < 0) return;
    const GbSplitPos SP = P.sps[spi];
    const int c0 = info.z * P.B, c1 = min(P.n, c0 + P.B), j = c0 + jl;
    if (j >= c1) return;
    auto meta = [&](int k, int& x, int& y, int& shift, unsigned& mask) {
        const int at = SP.jk0 + jl * P.n_sum + k;
        const int2 rg = P.jk[at];
        const GbJkD J = P.jkd[at];
        x = rg.x;
        y = rg.y;
        shift = J.shift;
        mask = J.mask;
    };
    int lo, nb;
    const bool fits = mv_bits(P.n_sum, meta, j - info.x, info.y, sp.mshift, lo, nb);
    if (kind == 0 && combo == 0 && Tb.mvb)
        Tb.mvb[(size_t)p * P.B + jl] = fits ? (unsigned short)(lo | nb << 8) : (unsigned short)0xffff;
    if (!fits || combo >= (1 << nb)) return;
    ChildCtx c;
    c.p = p;
    c.r = (unsigned)combo << lo;
    c.info = info;
    c.slot = par.slot[p];
    c.valid = true;
    const View<double> X64 = view64(pool, par, c, sp);
    const unsigned unit = P.outer_unit ? 0xffffffffu : 1u;
    const size_t at = (((size_t)p * P.B + jl) << GB_MV_BITS) + combo;
    if (kind == 0) {
        const iv64 g = tab_partial<double>(P, Tb, leaf_tab<double>(Tb, p), part_tab<double>(Tb, p), SP, j, c0, c.r,
                                           (const iv64*)nullptr, unit, ops64);
        Tb.mv64[at] = mono_hit(P, X64, j, gt_zero(g.lo), lt_zero(g.hi)) ? 1 : 0;
    } else {
        const iv32 g = tab_partial<float>(P, Tb, leaf_tab<float>(Tb, p), part_tab<float>(Tb, p), SP, j, c0, c.r,
                                          (const iv32*)nullptr, unit, ops32);
        Tb.mv32[at] = mono_hit(P, X64, j, gt_zero(g.lo), lt_zero(g.hi)) ? 1 : 0;
    }
}

template <typename T>
__device__ __forceinline__ bool tab_mono(const GbProg& P, const GbTabs& Tb, long long p, const GbSplitPos& SP,
                                         int blk, unsigned r, const View<double>& X64,
                                         const typename TabPrec<T>::I* O, typename TabPrec<T>::I* OA, int& ops) {
    typedef typename TabPrec<T>::I I;
    unsigned unit = 1u;   // a single outer sum: its adjoint is [1, 1]
    if (!P.outer_sum) {
        for (int t = 0; t < P.n_outer; t++) OA[t] = mk<T>((T)0, (T)0);
        OA[P.outer_root] = mk<T>((T)1, (T)1);
        reverse_sweep<T>(P.outer, P.n_outer, O, OA, ops);
        unit = unit_sums(P, OA);
    }
    const int c0 = blk * P.B, c1 = min(P.n, c0 + P.B);
    const typename TabPrec<T>::P2* tl = leaf_tab<T>(Tb, p);
    const typename TabPrec<T>::P2* td = part_tab<T>(Tb, p);
    for (int j = c0; j < c1; j++) {
        const I g = tab_partial<T>(P, Tb, tl, td, SP, j, c0, r, OA, unit, ops);
        if (mono_hit(P, X64, j, gt_zero(g.lo), lt_zero(g.hi))) return true;
    }
    return false;
}

// F and midpoint sums of a child in one walk over the term-tree segments.
__device__ __forceinline__ void tab_sums64(const GbProg& P, const GbTabs& Tb, long long p, const GbSplitPos& SP,
                                           int blk, unsigned r, iv64* sums, iv64* msums, int& ops) {
    const double2* tv = Tb.tv64 + (size_t)p * Tb.max_rows;
    const double2* tm = Tb.tm64 + (size_t)p * Tb.max_rows;
    const double2* ts = Tb.ts64 + (size_t)p * Tb.max_srows;
    const double2* tsm = Tb.tsm64 + (size_t)p * Tb.max_srows;
    const double2* nf = Tb.nf64 + (size_t)p * Tb.tree_nodes;
    const double2* nm = Tb.nm64 + (size_t)p * Tb.tree_nodes;
    int sg = SP.seg0;
    const int send = SP.seg0 + SP.nseg;
    for (int k = 0; k < P.n_sum; k++) {
        const GbSum S = P.sums[k];
        const int2 dr = P.dirty[blk * P.n_sum + k];
        iv64 curF[GB_TAB_MAX_DIRTY], curM[GB_TAB_MAX_DIRTY];
        for (int g = dr.x; g < dr.y; g++) {
            Tree<iv64> tf, tmid;
            tf.init();
            tmid.init();
            int ns = 0;
            while (sg < send) {
                const GbSeg G = P.segs[sg];
                if (G.sum != k || G.group != g) break;
                const int at = G.base + (int)((r >> G.shift) & G.mask);
                const double2 a = G.level ? ts[at] : tv[at], b = G.level ? tsm[at] : tm[at];
                tf.push_level(iv64{a.x, a.y}, G.level);
                tmid.push_level(iv64{b.x, b.y}, G.level);
                ns++;
                sg++;
            }
            ops += 4 * (ns > 0 ? ns - 1 : 0);
            curF[g - dr.x] = tf.result();
            curM[g - dr.x] = tmid.result();
        }
        const double2* nfk = nf + S.node0;
        const double2* nmk = nm + S.node0;
        auto nodeF = [&](int i) { const double2 v = nfk[i]; return iv64{v.x, v.y}; };
        auto nodeM = [&](int i) { const double2 v = nmk[i]; return iv64{v.x, v.y}; };
        sums[k] = tab_path(S, dr, curF, nodeF, ops);
        msums[k] = tab_path(S, dr, curM, nodeM, ops);
    }
}

// Register-resident forms of the single-sum walk, for objectives whose outer
// expression is one sum and whose blocks have at most GB_REG_DIRTY dirty
// groups of fewer than 2^GB_REG_LEVELS terms (checked on the host).  The
// level, count and range tests depend only on the parent's split position,
// so they are the same for every lane.  Every case of them (carries of a
// push, levels present, a path level's width) is its own straight-line
// code reached through a switch: array indices are constants, so nothing
// goes to thread-local memory, and no FP64 operation is issued under a
// false predicate (a warp's FP64 instruction holds the pipe whatever its
// active lanes).  Same operations in the same order as Tree, tab_path and
// tab_sums64, so the same sums.
static_assert(GB_REG_LEVELS == 5, "the switch cases below cover 5 levels");
static_assert(GB_REG_DIRTY == 4, "the switch cases below cover 4 dirty groups");
struct RegTree64 {
    iv64 lvl[GB_REG_LEVELS];
    unsigned cnt;
    __device__ __forceinline__ void init() { cnt = 0; }
    // v combined with the stored levels L .. L + K - 1 (lowest first), the
    // result stored at level L + K
    template <int L, int K>
    __device__ __forceinline__ void put(iv64 v) {
#pragma unroll
        for (int i = 0; i < K; i++) v = iadd(lvl[L + i], v);
        lvl[L + K] = v;
    }
    // Tree::push_level: the carries are the set bits of cnt from L up
    __device__ __forceinline__ void push_level(iv64 v, int L) {
        const int k = __ffs(~(cnt >> L)) - 1;
        switch (L * 8 + k) {
#define GB_PUT(a, b) \
    case (a) * 8 + (b): put<a, b>(v); break;
            GB_PUT(0, 0) GB_PUT(0, 1) GB_PUT(0, 2) GB_PUT(0, 3) GB_PUT(0, 4)
            GB_PUT(1, 0) GB_PUT(1, 1) GB_PUT(1, 2) GB_PUT(1, 3)
            GB_PUT(2, 0) GB_PUT(2, 1) GB_PUT(2, 2)
            GB_PUT(3, 0) GB_PUT(3, 1)
            GB_PUT(4, 0)
#undef GB_PUT
            default: break;   // beyond the levels the host check allows
        }
        cnt += 1u << L;
    }
    // Tree::result for the levels present M (ascending order)
    template <unsigned M>
    __device__ __forceinline__ iv64 res() const {
        iv64 r{0.0, 0.0};
        bool have = false;
#pragma unroll
        for (int i = 0; i < GB_REG_LEVELS; i++) {
            if ((M >> i) & 1u) {
                r = have ? iadd(lvl[i], r) : lvl[i];
                have = true;
            }
        }
        return r;
    }
    __device__ __forceinline__ iv64 result() const {
        switch (cnt) {
#define GB_RES(m) \
    case m: return res<m>();
            GB_RES(1) GB_RES(2) GB_RES(3) GB_RES(4) GB_RES(5) GB_RES(6) GB_RES(7) GB_RES(8)
            GB_RES(9) GB_RES(10) GB_RES(11) GB_RES(12) GB_RES(13) GB_RES(14) GB_RES(15) GB_RES(16)
            GB_RES(17) GB_RES(18) GB_RES(19) GB_RES(20) GB_RES(21) GB_RES(22) GB_RES(23) GB_RES(24)
            GB_RES(25) GB_RES(26) GB_RES(27) GB_RES(28) GB_RES(29) GB_RES(30) GB_RES(31)
#undef GB_RES
            default: return iv64{0.0, 0.0};   // empty
        }
    }
};

// One level of tab_path over NT parents (SINGLE: the last one has no right
// child).  Node a of the level below sits at cur[a - lo]; the t-th parent's
// children a = 2(nlo + t), a + 1 sit at 2t - (lo & 1) and 2t + 1 - (lo & 1),
// both at or after t, so the level is rebuilt in place in ascending t.
template <int NT, bool SINGLE, typename N>
__device__ __forceinline__ void path_level(iv64 (&cur)[GB_REG_DIRTY], int lo, int hi, int nlo, int off, N node,
                                           int& ops) {
    const bool odd = lo & 1;
#pragma unroll
    for (int t = 0; t < NT; t++) {
        const int a = 2 * (nlo + t);
        constexpr int D = GB_REG_DIRTY - 1;
        const int e0 = 2 * t, e1 = 2 * t + 1;   // even lo: cur indices of a, a + 1
        const iv64 ca = odd ? cur[e0 - 1 < 0 ? 0 : (e0 - 1 > D ? D : e0 - 1)] : cur[e0 > D ? D : e0];
        const iv64 left = (a >= lo && a < hi) ? ca : node(off + a);
        if (SINGLE && t == NT - 1) {
            cur[t] = left;
        } else {
            const iv64 cb = odd ? cur[e1 - 1 > D ? D : e1 - 1] : cur[e1 > D ? D : e1];
            const iv64 right = (a + 1 >= lo && a + 1 < hi) ? cb : node(off + a + 1);
            cur[t] = iadd(left, right);
            ops += 2;
        }
    }
}

// tab_path over at most GB_REG_DIRTY dirty nodes per level.
template <typename N>
__device__ __forceinline__ iv64 tab_path_reg(const GbSum& S, int2 dr, iv64 (&cur)[GB_REG_DIRTY], N node, int& ops) {
    if (S.ngroups == 0 || S.nnodes <= 0) return iv64{0.0, 0.0};
    int lo = dr.x, hi = dr.y, off = 0;
    if (lo >= hi) return node(S.nnodes - 1);   // no dirty group: the parent's root
    for (int mL = S.ngroups; mL > 1; mL = (mL + 1) / 2) {
        const int nlo = lo >> 1, nhi = ((hi - 1) >> 1) + 1;
        const bool single = 2 * (nhi - 1) + 1 >= mL;
        switch ((nhi - nlo) * 2 + (single ? 1 : 0)) {
            case 2: path_level<1, false>(cur, lo, hi, nlo, off, node, ops); break;
            case 3: path_level<1, true>(cur, lo, hi, nlo, off, node, ops); break;
            case 4: path_level<2, false>(cur, lo, hi, nlo, off, node, ops); break;
            case 5: path_level<2, true>(cur, lo, hi, nlo, off, node, ops); break;
            case 6: path_level<3, false>(cur, lo, hi, nlo, off, node, ops); break;
            case 7: path_level<3, true>(cur, lo, hi, nlo, off, node, ops); break;
            case 8: path_level<4, false>(cur, lo, hi, nlo, off, node, ops); break;
            case 9: path_level<4, true>(cur, lo, hi, nlo, off, node, ops); break;
            default: break;   // wider than the host check allows
        }
        lo = nlo;
        hi = nhi;
        off += mL;
    }
    return cur[0];
}

// The one sum of a child over the box (MID false) or at its midpoint (MID
// true): its dirty groups from the term-tree segments, then the group-tree
// path (tab_sums64 for n_sum = 1, one of its two walks).
template <bool MID>
__device__ __forceinline__ iv64 tab_sum1_reg(const GbProg& P, const GbTabs& Tb, long long p, const GbSplitPos& SP,
                                             int blk, unsigned r, int& ops) {
    const double2* tv = (MID ? Tb.tm64 : Tb.tv64) + (size_t)p * Tb.max_rows;
    const double2* ts = (MID ? Tb.tsm64 : Tb.ts64) + (size_t)p * Tb.max_srows;
    const double2* nd = (MID ? Tb.nm64 : Tb.nf64) + (size_t)p * Tb.tree_nodes;
    const GbSum S = P.sums[0];
    const int2 dr = P.dirty[blk];
    iv64 cur[GB_REG_DIRTY];
    int sg = SP.seg0;
    const int send = SP.seg0 + SP.nseg;
#pragma unroll
    for (int t = 0; t < GB_REG_DIRTY; t++) {
        cur[t] = iv64{0.0, 0.0};
        const int g = dr.x + t;
        if (g < dr.y) {
            RegTree64 tr;
            tr.init();
            int ns = 0;
            while (sg < send) {
                const GbSeg G = P.segs[sg];
                if (G.sum != 0 || G.group != g) break;
                const int at = G.base + (int)((r >> G.shift) & G.mask);
                const double2 a = G.level ? ts[at] : tv[at];
                tr.push_level(iv64{a.x, a.y}, G.level);
                ns++;
                sg++;
            }
            ops += 2 * (ns > 0 ? ns - 1 : 0);
            cur[t] = tr.result();
        }
    }
    const double2* ndk = nd + S.node0;
    return tab_path_reg(S, dr, cur, [&](int i) { const double2 v = ndk[i]; return iv64{v.x, v.y}; }, ops);
}

// FP64 child: midpoint sample, F(X), cut-off.  SUM1: the outer expression
// is one sum (F is that sum; the first-order test is left to
// eval64_tab_mono and *need_mono tells whether the child passed the
// cut-off).  Otherwise the first-order test follows at once and the flag is
// set here.  Returns false for an invalid child.
template <bool SUM1, bool REG = false>
__device__ __forceinline__ bool eval64_tab_child(const GbProg& P, const GbPool& pool, const GbParents& par,
                                                 const GbTabs& Tb, const GbChildren& ch, long long ci,
                                                 const GbSplit& sp, double gub_prev, unsigned long long* gkey,
                                                 bool* has_key, int& ops, bool* need_mono) {
    ChildCtx c = child_ctx(par, ci, sp);
    const int spi = c.valid ? P.sp_of_cyc[c.info.x] : -1;
    *need_mono = false;
    if (spi < 0) {   // invalid child (or, defensively, a split position without a layout)
        ch.flag[ci] = 0;
        ch.flo[ci] = __longlong_as_double(0x7ff0000000000000LL);
        return false;
    }
    const GbSplitPos SP = P.sps[spi];
    const int blk = c.info.z;
    if constexpr (SUM1 && REG) {
        const iv64 F = tab_sum1_reg<false>(P, Tb, c.p, SP, blk, c.r, ops);
        const iv64 Fm = tab_sum1_reg<true>(P, Tb, c.p, SP, blk, c.r, ops);
        if (Fm.hi == Fm.hi) {
            *gkey = gb_order_key(Fm.hi);
            *has_key = true;
        }
        const bool keep = !(F.lo > gub_prev);
        ch.flo[ci] = canon_lo(F.lo);
        if (keep) *need_mono = true;
        else ch.flag[ci] = 0;
        return true;
    }
    View<double> X = view64(pool, par, c, sp);
    iv64 sums[GB_MAX_ISUM], msums[GB_MAX_ISUM];
    tab_sums64(P, Tb, c.p, SP, blk, c.r, sums, msums, ops);
    if constexpr (SUM1) {
        const iv64 Fm = msums[0], F = sums[0];
        if (Fm.hi == Fm.hi) {
            *gkey = gb_order_key(Fm.hi);
            *has_key = true;
        }
        const bool keep = !(F.lo > gub_prev);
        ch.flo[ci] = canon_lo(F.lo);
        if (keep) *need_mono = true;
        else ch.flag[ci] = 0;
    } else {
        MidView MX{X};
        iv64 O[GB_MAX_OREGS], OA[GB_MAX_OREGS];
        iv64 Fm = outer_value<double>(P, MX, msums, O, ops);
        if (Fm.hi == Fm.hi) {
            *gkey = gb_order_key(Fm.hi);
            *has_key = true;
        }
        iv64 F = outer_value<double>(P, X, sums, O, ops);
        bool keep = !(F.lo > gub_prev);
        ch.flo[ci] = canon_lo(F.lo);
        if (keep) keep = !tab_mono<double>(P, Tb, c.p, SP, blk, c.r, X, O, OA, ops);
        ch.flag[ci] = keep ? 1 : 0;
    }
    return true;
}

// First-order test of a child that passed the cut-off, for objectives whose
// outer expression is one sum (its adjoint is [1, 1], so the test needs no
// outer values); sets the child's flag.
__device__ __forceinline__ void eval64_tab_mono(const GbProg& P, const GbPool& pool, const GbParents& par,
                                                const GbTabs& Tb, const GbChildren& ch, long long ci,
                                                const GbSplit& sp, int& ops) {
    const ChildCtx c = child_ctx(par, ci, sp);
    const GbSplitPos SP = P.sps[P.sp_of_cyc[c.info.x]];
    const View<double> X = view64(pool, par, c, sp);
    iv64 O[1], OA[1];
    const bool mono = tab_mono<double>(P, Tb, c.p, SP, c.info.z, c.r, X, O, OA, ops);
    ch.flag[ci] = mono ? 0 : 1;
}

// eval64_tab_mono for one sum (n_sum = 1, no outer VAR leaves): its
// adjoint is [1, 1], so each partial is the tabulated sum alone.
__device__ __forceinline__ void eval64_tab_mono1(const GbProg& P, const GbPool& pool, const GbParents& par,
                                                 const GbTabs& Tb, const GbChildren& ch, long long ci,
                                                 const GbSplit& sp, int& ops) {
    const ChildCtx c = child_ctx(par, ci, sp);
    const GbSplitPos SP = P.sps[P.sp_of_cyc[c.info.x]];
    const View<double> X = view64(pool, par, c, sp);
    const int c0 = c.info.z * P.B, c1 = min(P.n, c0 + P.B);
    const double2* tl = leaf_tab<double>(Tb, c.p);
    const double2* td = part_tab<double>(Tb, c.p);
    bool mono = false;
    for (int j = c0; j < c1 && !mono; j++) {
        const iv64 g = tab_partial<double>(P, Tb, tl, td, SP, j, c0, c.r, (const iv64*)nullptr, 1u, ops);
        mono = mono_hit(P, X, j, gt_zero(g.lo), lt_zero(g.hi));
    }
    ch.flag[ci] = mono ? 0 : 1;
}

// One child per thread.  When the outer expression is one sum, the children
// of a warp that pass the cut-off are queued in shared memory and their
// first-order tests run 32 at a time, every lane busy, instead of inside the
// branch of the lanes that passed (the same tests, so the same flags).
template <bool QUEUE, bool REG>
__global__ void __launch_bounds__(128, REG ? GB_TAB_MINB_REG : GB_TAB_MINB) k_eval64_tab(GbProg P, GbPool pool, GbParents par, GbTabs Tb,
                                                    GbChildren ch, GbSplit sp, int from_list, GbState* st) {
    gb_grid_trigger();
    gb_grid_wait();
    if (st->halt) return;
    __shared__ unsigned s_queue[4][QUEUE ? 64 : 1];   // per warp: at most 31 left over + 32 new
    const long long lim = from_list ? st->n32 : st->nch;
    const double gub_prev = gb_key_value(st->gub_key);
    const long long stride = (long long)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    unsigned* q = s_queue[threadIdx.x >> 5];
    constexpr bool queue = QUEUE;
    int qn = 0;   // warp-uniform queue length
    int ops = 0;
    unsigned long long key = ~0ull, nvalid = 0;
    bool has = false;
    for (long long base = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); base < lim; base += stride) {
        const long long idx = base + lane;
        bool valid = false, need = false;
        long long ci = 0;
        if (idx < lim) {
            ci = from_list ? (long long)ch.list32[idx] : idx;
            unsigned long long k2 = ~0ull;
            bool h2 = false;
            valid = eval64_tab_child<QUEUE, REG>(P, pool, par, Tb, ch, ci, sp, gub_prev, &k2, &h2, ops, &need);
            if (h2 && k2 < key) key = k2, has = true;
        }
        nvalid += __popc(__ballot_sync(0xffffffffu, valid));
        if constexpr (!queue) continue;
        const unsigned bal = __ballot_sync(0xffffffffu, need);
        if (need) q[qn + __popc(bal & ((1u << lane) - 1u))] = (unsigned)ci;
        qn += __popc(bal);
        __syncwarp();
        if (qn >= 32) {
            if constexpr (REG) eval64_tab_mono1(P, pool, par, Tb, ch, q[qn - 32 + lane], sp, ops);
            else eval64_tab_mono(P, pool, par, Tb, ch, q[qn - 32 + lane], sp, ops);
            qn -= 32;
            __syncwarp();
        }
    }
    if (queue && lane < qn) {   // the rest of the queue
        if constexpr (REG) eval64_tab_mono1(P, pool, par, Tb, ch, q[lane], sp, ops);
        else eval64_tab_mono(P, pool, par, Tb, ch, q[lane], sp, ops);
    }
    warp_min_gub(key, has, st);
    warp_add_ops(ops, &st->ops64);
    if (lane == 0 && nvalid) {
        atomicAdd((unsigned long long*)&st->evals64, nvalid);
        atomicAdd((unsigned long long*)&st->mids, nvalid);
        if (!from_list) atomicAdd((unsigned long long*)&st->children, nvalid);
    }
}

__global__ void __launch_bounds__(128, GB_TAB_MINB) k_eval32_tab(GbProg P, GbPool pool, GbParents par, GbTabs Tb,
                                                    GbChildren ch, GbSplit sp, GbState* st) {
    if (st->halt) return;
    const long long lim = st->nch;
    const double gub_prev = gb_key_value(st->gub_key);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); base < lim; base += stride) {
        long long ci = base + (threadIdx.x & 31);
        bool valid = false;
        int ops = 0;
        if (ci < lim) {
            ChildCtx c = child_ctx(par, ci, sp);
            ch.flag[ci] = 0;
            ch.flo[ci] = __longlong_as_double(0x7ff0000000000000LL);
            const int spi = c.valid ? P.sp_of_cyc[c.info.x] : -1;
            if (spi >= 0) {
                valid = true;
                const GbSplitPos SP = P.sps[spi];
                const int blk = c.info.z;
                View<float> X = view32(pool, par, c, sp);
                View<double> X64 = view64(pool, par, c, sp);
                iv32 O[GB_MAX_OREGS], OA[GB_MAX_OREGS], sums[GB_MAX_ISUM];
                int sg = SP.seg0;
                for (int k = 0; k < P.n_sum; k++)
                    sums[k] = tab_sum32(P, Tb, c.p, SP, k, blk, c.r, sg, ops);
                iv32 F = outer_value<float>(P, X, sums, O, ops);
                bool keep = !((double)F.lo > gub_prev);
                if (keep) keep = !tab_mono<float>(P, Tb, c.p, SP, blk, c.r, X64, O, OA, ops);
                ch.flag32[ci] = keep ? 1 : 0;
            } else {
                ch.flag32[ci] = 0;
            }
        }
        warp_add_ops(ops, &st->ops32);
        unsigned nv = __popc(__ballot_sync(0xffffffffu, valid));
        if ((threadIdx.x & 31) == 0 && nv) {
            atomicAdd((unsigned long long*)&st->evals32, (unsigned long long)nv);
            atomicAdd((unsigned long long*)&st->children, (unsigned long long)nv);
        }
    }
}

// ---------------------------------------------------------------------------
// One child per warp (generations with few children): the lanes share the
// dirty terms of each group (warp_group) and the coordinates of the
// first-order test; the group-tree paths and the outer expression are
// computed by every lane alike.  Same operations in the same order as the
// per-thread kernels, so the results are identical.  Operation counts: the
// work every lane repeats is counted once (lane 0), the shared work per lane.

// The partial-table entries of a split position's block, (coordinate,
// sum)-major, staged in shared memory by the warp that evaluates a child:
// jk range, partial-table base and digit field (shift | mask << 16).
constexpr int GB_WMETA = 384;
struct WMeta { int x, y, base, sm; };

// Per-warp shared scratch of the one-child-per-warp kernels: the outer
// expression's values and adjoints (written by lane 0, read by every lane
// in the first-order test) and the staged partial-table entries.
struct WScratch {
    iv64* O64;
    iv64* OA64;
    iv32* O32;
    iv32* OA32;
    WMeta* meta;
};
template <typename T> __device__ __forceinline__ typename TabPrec<T>::I* ws_O(const WScratch& w);
template <> __device__ __forceinline__ iv64* ws_O<double>(const WScratch& w) { return w.O64; }
template <> __device__ __forceinline__ iv32* ws_O<float>(const WScratch& w) { return w.O32; }
template <typename T> __device__ __forceinline__ typename TabPrec<T>::I* ws_OA(const WScratch& w);
template <> __device__ __forceinline__ iv64* ws_OA<double>(const WScratch& w) { return w.OA64; }
template <> __device__ __forceinline__ iv32* ws_OA<float>(const WScratch& w) { return w.OA32; }

// The kernels' shared declarations: 4 warps per block.
#define GB_WSCRATCH_DECL                                                   \
    __shared__ WMeta s_meta[4][GB_WMETA];                                  \
    __shared__ iv64 s_o64[4][GB_MAX_OREGS], s_oa64[4][GB_MAX_OREGS];       \
    __shared__ iv32 s_o32[4][GB_MAX_OREGS], s_oa32[4][GB_MAX_OREGS];       \
    const int wib_ = threadIdx.x >> 5;                                     \
    const WScratch ws{s_o64[wib_], s_oa64[wib_], s_o32[wib_], s_oa32[wib_], s_meta[wib_]};

__device__ __forceinline__ bool stage_meta(const GbProg& P, const GbSplitPos& SP, int cnt, WMeta* m, int lane) {
    if (cnt > GB_WMETA) return false;
    // up to 4 entries per lane in flight at once (one memory round trip per 128 entries)
    for (int e0 = 0; e0 < cnt; e0 += 128) {
        int2 rg[4];
        GbJkD J[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int e = e0 + u * 32 + lane;
            if (e < cnt) {
                rg[u] = P.jk[SP.jk0 + e];
                J[u] = P.jkd[SP.jk0 + e];
            }
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int e = e0 + u * 32 + lane;
            if (e < cnt) m[e] = WMeta{rg[u].x, rg[u].y, J[u].base, (int)(unsigned short)J[u].shift | ((int)J[u].mask << 16)};
        }
    }
    __syncwarp();
    return true;
}

// tab_partial from the staged entries: the tabulated sums of every sum are
// loaded together (one round of memory latency), then combined in the same
// order as tab_partial.
template <typename T>
__device__ __forceinline__ typename TabPrec<T>::I tab_partial_m(const GbProg& P, const GbTabs& Tb,
                                                                const typename TabPrec<T>::P2* tl,
                                                                const typename TabPrec<T>::P2* td, const WMeta* M,
                                                                int j, int c0, unsigned r,
                                                                const typename TabPrec<T>::I* OA, unsigned unit,
                                                                int& ops) {
    typedef typename TabPrec<T>::I I;
    typedef typename TabPrec<T>::P2 P2;
    const WMeta* mj = M + (j - c0) * P.n_sum;
    P2 e[GB_MAX_ISUM];
#pragma unroll
    for (int k = 0; k < GB_MAX_ISUM; k++) {
        if (k < P.n_sum) {
            const WMeta m = mj[k];
            const int shift = (short)(m.sm & 0xffff);
            if (m.x != m.y && shift >= 0) e[k] = td[m.base + (int)((r >> shift) & ((unsigned)m.sm >> 16))];
        }
    }
    I g;
    bool have = false;
    for (int v = 0; v < P.n_var_leaves; v++) {
        GbVarLeaf L = P.var_leaves[v];
        if (L.coord != j) continue;
        if (have) g = iadd(g, OA[L.reg]), ops += 2;
        else g = OA[L.reg], have = true;
    }
#pragma unroll
    for (int k = 0; k < GB_MAX_ISUM; k++) {
        if (k >= P.n_sum) break;
        const WMeta m = mj[k];
        if (m.x == m.y) continue;
        const int shift = (short)(m.sm & 0xffff);
        I Dk;
        if (shift >= 0) {
            Dk = mk<T>(e[k].x, e[k].y);
        } else {
            for (int q = m.x; q < m.y; q++) {
                const GbContrib C = P.contribs[q];
                const unsigned combo = (r >> C.dshift) & C.mask;
                const P2 t = tl[C.base + (int)combo * Tb.max_leaves];
                const I v = mk<T>(t.x, t.y);
                if (q > m.x) Dk = iadd(Dk, v), ops += 2;
                else Dk = v;
            }
        }
        I term;
        if ((unit >> k) & 1u) term = Dk;
        else term = imul(OA[P.sums[k].outer_reg], Dk), ops += 2;
        if (have) g = iadd(g, term), ops += 2;
        else g = term, have = true;
    }
    if (!have) g = mk<T>((T)0, (T)0);
    return g;
}

// First-order test, coordinates of the block spread over the lanes (the
// block's partial-table entries staged in shared memory when they fit).
// The outer adjoints are computed by lane 0 from the outer values in the
// warp's scratch and shared through it.
template <typename T>
__device__ __forceinline__ bool tab_mono_w(const GbProg& P, const GbTabs& Tb, long long p, const GbSplitPos& SP,
                                           int blk, unsigned r, const View<double>& X64, const WScratch& ws,
                                           int& red, int& par, int lane) {
    typedef typename TabPrec<T>::I I;
    I* O = ws_O<T>(ws);
    I* OA = ws_OA<T>(ws);
    unsigned unit = P.outer_unit ? 0xffffffffu : 1u;   // a single outer sum: its adjoint is [1, 1]
    if (!P.outer_sum && !P.outer_unit) {
        if (lane == 0) {
            for (int t = 0; t < P.n_outer; t++) OA[t] = mk<T>((T)0, (T)0);
            OA[P.outer_root] = mk<T>((T)1, (T)1);
            reverse_sweep<T>(P.outer, P.n_outer, O, OA, red);
            unit = unit_sums(P, OA);
        }
        __syncwarp();
        unit = __shfl_sync(0xffffffffu, unit, 0);
    }
    const int c0 = blk * P.B, c1 = min(P.n, c0 + P.B);
    const typename TabPrec<T>::P2* tl = leaf_tab<T>(Tb, p);
    const typename TabPrec<T>::P2* td = part_tab<T>(Tb, p);
    bool hit = false;
    const unsigned char* mvt = sizeof(T) == 8 ? Tb.mv64 : Tb.mv32;
    if (mvt && Tb.mvb) {   // the parent's digit fields: one lookup per coordinate when all have a table
        bool all = true;
        for (int j = c0 + lane; j < c1; j += 32) {
            const unsigned e = Tb.mvb[(size_t)p * P.B + (j - c0)];
            if (e == 0xffffu) {
                all = false;
                continue;
            }
            const unsigned lo = e & 0xffu, nb = e >> 8;
            hit |= mvt[(((size_t)p * P.B + (j - c0)) << GB_MV_BITS) + ((r >> lo) & ((1u << nb) - 1u))] != 0;
        }
        if (__all_sync(0xffffffffu, all)) return __any_sync(0xffffffffu, hit);
        hit = false;   // some coordinate has no table: the test below covers every coordinate
    }
    if (stage_meta(P, SP, (c1 - c0) * P.n_sum, ws.meta, lane)) {
        // the parent's verdict table where the coordinate has one (mono_fill)
        const unsigned char* mv = sizeof(T) == 8 ? Tb.mv64 : Tb.mv32;
        for (int j = c0 + lane; j < c1; j += 32) {
            int lo, nb;
            const WMeta* mj = ws.meta + (j - c0) * P.n_sum;
            auto meta = [&](int k, int& x, int& y, int& shift, unsigned& mask) {
                const WMeta m = mj[k];
                x = m.x;
                y = m.y;
                shift = (short)(m.sm & 0xffff);
                mask = (unsigned)m.sm >> 16;
            };
            if (mv && mv_bits(P.n_sum, meta, j - X64.c0, X64.dd, X64.mshift, lo, nb)) {
                hit |= mv[(((size_t)p * P.B + (j - c0)) << GB_MV_BITS) + ((r >> lo) & ((1u << nb) - 1u))] != 0;
                continue;
            }
            const I g = tab_partial_m<T>(P, Tb, tl, td, ws.meta, j, c0, r, OA, unit, par);
            hit |= mono_hit(P, X64, j, gt_zero(g.lo), lt_zero(g.hi));
        }
    } else {
        for (int j = c0 + lane; j < c1 && !hit; j += 32) {
            const I g = tab_partial<T>(P, Tb, tl, td, SP, j, c0, r, OA, unit, par);
            hit = mono_hit(P, X64, j, gt_zero(g.lo), lt_zero(g.hi));
        }
    }
    __syncwarp();   // the scratch is reused by the warp's next child
    return __any_sync(0xffffffffu, hit);
}

// F from lane 0's sums (the outer expression evaluated by lane 0 into the
// warp's scratch), broadcast to every lane.
template <typename T, typename V>
__device__ __forceinline__ typename TabPrec<T>::I outer_w(const GbProg& P, const V& X,
                                                          const typename TabPrec<T>::I* sums, const WScratch& ws,
                                                          int lane, int& red) {
    typedef typename TabPrec<T>::I I;
    I F{};
    if (lane == 0) F = outer_value<T>(P, X, sums, ws_O<T>(ws), red);
    __syncwarp();
    F.lo = __shfl_sync(0xffffffffu, F.lo, 0);
    F.hi = __shfl_sync(0xffffffffu, F.hi, 0);
    return F;
}

__device__ __forceinline__ bool eval64_tab_child_w(const GbProg& P, const GbPool& pool, const GbParents& par,
                                                   const GbTabs& Tb, const GbChildren& ch, long long ci,
                                                   const GbSplit& sp, double gub_prev, unsigned long long* gkey,
                                                   bool* has_key, int& red, int& pops, int lane, const WScratch& ws) {
    const ChildCtx c = child_ctx(par, ci, sp);
    const int spi = c.valid ? P.sp_of_cyc[c.info.x] : -1;
    if (spi < 0) {
        if (lane == 0) {
            ch.flag[ci] = 0;
            ch.flo[ci] = __longlong_as_double(0x7ff0000000000000LL);
        }
        return false;
    }
    const GbSplitPos SP = P.sps[spi];
    const int blk = c.info.z;
    const View<double> X = view64(pool, par, c, sp);
    const MidView MX{X};
    const size_t rowbase = (size_t)c.p * Tb.max_rows, nbase = (size_t)c.p * Tb.tree_nodes;
    const size_t sbase = (size_t)c.p * Tb.max_srows;
    iv64 sums[GB_MAX_ISUM], msums[GB_MAX_ISUM];   // lane 0's
    int dt = SP.seg0;
    if (Tb.cs64) {   // computed by k_child_sums
        if (lane == 0)
            for (int k = 0; k < P.n_sum; k++) {
                const double2 a = Tb.cs64[(size_t)ci * P.n_sum + k], b = Tb.csm64[(size_t)ci * P.n_sum + k];
                sums[k] = iv64{a.x, a.y};
                msums[k] = iv64{b.x, b.y};
            }
    } else
    for (int k = 0; k < P.n_sum; k++) {
        const GbSum S = P.sums[k];
        const int2 dr = P.dirty[blk * P.n_sum + k];
        iv64 curF[GB_TAB_MAX_DIRTY], curM[GB_TAB_MAX_DIRTY];
        for (int g = dr.x; g < dr.y; g++) {
            iv64 v2[2];
            int cnt;
            warp_group<iv64, 2>(P, SP, k, g, c.r, dt, lane,
                                [&](const GbSeg& G, int at, iv64* v) {
                                    const double2 a = G.level ? Tb.ts64[sbase + at] : Tb.tv64[rowbase + at];
                                    const double2 b = G.level ? Tb.tsm64[sbase + at] : Tb.tm64[rowbase + at];
                                    v[0] = iv64{a.x, a.y};
                                    v[1] = iv64{b.x, b.y};
                                }, v2, cnt);
            if (lane == 0) {
                curF[g - dr.x] = v2[0];
                curM[g - dr.x] = v2[1];
            }
            red += 4 * (cnt > 0 ? cnt - 1 : 0);
        }
        const size_t nb = nbase + S.node0;
        const iv64 a = tab_path_w(S, dr, curF, [&](int i) { return TabPrec<double>::node(Tb, nb + i); }, lane, red);
        const iv64 b = tab_path_w(S, dr, curM, [&](int i) { return mid_node(Tb, nb + i); }, lane, red);
        if (lane == 0) sums[k] = a, msums[k] = b;
    }
    const iv64 Fm = outer_w<double>(P, MX, msums, ws, lane, red);
    if (lane == 0 && Fm.hi == Fm.hi) {
        *gkey = gb_order_key(Fm.hi);
        *has_key = true;
    }
    const iv64 F = outer_w<double>(P, X, sums, ws, lane, red);   // leaves the outer values of X in the scratch
    bool keep = !(F.lo > gub_prev);   // the same in every lane
    if (keep) keep = !tab_mono_w<double>(P, Tb, c.p, SP, blk, c.r, X, ws, red, pops, lane);
    if (lane == 0) {
        ch.flo[ci] = canon_lo(F.lo);
        ch.flag[ci] = keep ? 1 : 0;
    }
    return true;
}

__global__ void __launch_bounds__(128, 1) k_eval64_tabw(GbProg P, GbPool pool, GbParents par, GbTabs Tb,
                                                     GbChildren ch, GbSplit sp, int from_list, GbState* st) {
    if (st->halt) return;
    const long long lim = from_list ? st->n32 : st->nch;
    const double gub_prev = gb_key_value(st->gub_key);
    const int lane = threadIdx.x & 31;
    GB_WSCRATCH_DECL
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    unsigned long long key = ~0ull;
    bool has = false;
    int red = 0, pops = 0;
    unsigned long long nv = 0;
    for (long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; w < lim; w += nw) {
        const long long ci = from_list ? (long long)ch.list32[w] : w;
        unsigned long long k2 = ~0ull;
        bool h2 = false;
        if (eval64_tab_child_w(P, pool, par, Tb, ch, ci, sp, gub_prev, &k2, &h2, red, pops, lane, ws)) nv++;
        if (h2 && k2 < key) key = k2, has = true;
    }
    warp_min_gub(key, has, st);
    warp_add_ops((lane == 0 ? red : 0) + pops, &st->ops64);
    if (lane == 0 && nv) {
        atomicAdd((unsigned long long*)&st->evals64, nv);
        atomicAdd((unsigned long long*)&st->mids, nv);
        if (!from_list) atomicAdd((unsigned long long*)&st->children, nv);
    }
}

// FP32 pass of one child by a warp: writes flag32 (and resets the FP64 flag
// and LB); returns -1 for an invalid child, else whether the child passed.
__device__ __forceinline__ int eval32_tab_child_w(const GbProg& P, const GbPool& pool, const GbParents& par,
                                                  const GbTabs& Tb, const GbChildren& ch, long long ci,
                                                  const GbSplit& sp, double gub_prev, int& red, int& pops,
                                                  int lane, const WScratch& ws) {
    const ChildCtx c = child_ctx(par, ci, sp);
    const int spi = c.valid ? P.sp_of_cyc[c.info.x] : -1;
    if (lane == 0) {
        ch.flag[ci] = 0;
        ch.flo[ci] = __longlong_as_double(0x7ff0000000000000LL);
    }
    if (spi < 0) {
        if (lane == 0) ch.flag32[ci] = 0;
        return -1;
    }
    const GbSplitPos SP = P.sps[spi];
    const int blk = c.info.z;
    const View<float> X = view32(pool, par, c, sp);
    const View<double> X64 = view64(pool, par, c, sp);
    const size_t rowbase = (size_t)c.p * Tb.max_rows, nbase = (size_t)c.p * Tb.tree_nodes;
    const size_t sbase = (size_t)c.p * Tb.max_srows;
    iv32 sums[GB_MAX_ISUM];   // lane 0's
    int dt = SP.seg0;
    if (Tb.cs32) {   // computed by k_child_sums
        if (lane == 0)
            for (int k = 0; k < P.n_sum; k++) {
                const float2 a = Tb.cs32[(size_t)ci * P.n_sum + k];
                sums[k] = iv32{a.x, a.y};
            }
    } else
    for (int k = 0; k < P.n_sum; k++) {
        const GbSum S = P.sums[k];
        const int2 dr = P.dirty[blk * P.n_sum + k];
        iv32 cur[GB_TAB_MAX_DIRTY];
        for (int g = dr.x; g < dr.y; g++) {
            int cnt;
            iv32 v;
            warp_group<iv32, 1>(P, SP, k, g, c.r, dt, lane,
                                [&](const GbSeg& G, int at, iv32* v) {
                                    const float2 a = G.level ? Tb.ts32[sbase + at] : Tb.tv32[rowbase + at];
                                    v[0] = iv32{a.x, a.y};
                                }, &v, cnt);
            if (lane == 0) cur[g - dr.x] = v;
            red += 2 * (cnt > 0 ? cnt - 1 : 0);
        }
        const size_t nb = nbase + S.node0;
        const iv32 a = tab_path_w(S, dr, cur, [&](int i) { return TabPrec<float>::node(Tb, nb + i); }, lane, red);
        if (lane == 0) sums[k] = a;
    }
    const iv32 F = outer_w<float>(P, X, sums, ws, lane, red);
    bool keep = !((double)F.lo > gub_prev);   // the same in every lane
    if (keep) keep = !tab_mono_w<float>(P, Tb, c.p, SP, blk, c.r, X64, ws, red, pops, lane);
    if (lane == 0) ch.flag32[ci] = keep ? 1 : 0;
    return keep ? 1 : 0;
}

__global__ void __launch_bounds__(128) k_eval32_tabw(GbProg P, GbPool pool, GbParents par, GbTabs Tb,
                                                     GbChildren ch, GbSplit sp, GbState* st) {
    if (st->halt) return;
    const long long lim = st->nch;
    const double gub_prev = gb_key_value(st->gub_key);
    const int lane = threadIdx.x & 31;
    GB_WSCRATCH_DECL
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    int red = 0, pops = 0;
    unsigned long long nv = 0;
    for (long long ci = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; ci < lim; ci += nw)
        if (eval32_tab_child_w(P, pool, par, Tb, ch, ci, sp, gub_prev, red, pops, lane, ws) >= 0) nv++;
    warp_add_ops((lane == 0 ? red : 0) + pops, &st->ops32);
    if (lane == 0 && nv) {
        atomicAdd((unsigned long long*)&st->evals32, nv);
        atomicAdd((unsigned long long*)&st->children, nv);
    }
}

// FP32 prefilter and FP64 evaluation in one pass, one child per warp: a warp
// whose child passes the FP32 test evaluates it in FP64 at once (the same
// children, the same previous GUB and the same operations as the FP32 kernel,
// the survivor list and the FP64 kernel in sequence, without the list).
// With `cc` (at most 2^16 children) the last block to finish lists the
// generation's survivors against the final incumbent (k_cc_small's work).
__global__ void __launch_bounds__(128, 1) k_eval3264_tabw(GbProg P, GbPool pool, GbParents par, GbTabs Tb,
                                                       GbChildren ch, GbSplit sp, GbState* st, GbGenConst G,
                                                       int cc) {
    gb_grid_trigger();
    gb_grid_wait();
    if (st->halt) return;
    const long long lim = st->nch;
    const double gub_prev = gb_key_value(st->gub_key);
    const int lane = threadIdx.x & 31;
    GB_WSCRATCH_DECL
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    int red32 = 0, pops32 = 0, red64 = 0, pops64 = 0;
    unsigned long long nv = 0, n32 = 0, key = ~0ull;
    bool has = false;
    for (long long ci = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; ci < lim; ci += nw) {
        const int v = eval32_tab_child_w(P, pool, par, Tb, ch, ci, sp, gub_prev, red32, pops32, lane, ws);
        if (v < 0) continue;
        nv++;
        if (v == 0) continue;
        n32++;
        unsigned long long k2 = ~0ull;
        bool h2 = false;
        eval64_tab_child_w(P, pool, par, Tb, ch, ci, sp, gub_prev, &k2, &h2, red64, pops64, lane, ws);
        if (h2 && k2 < key) key = k2, has = true;
    }
    warp_min_gub(key, has, st);
    warp_add_ops((lane == 0 ? red32 : 0) + pops32, &st->ops32);
    warp_add_ops((lane == 0 ? red64 : 0) + pops64, &st->ops64);
    if (lane == 0 && nv) {
        atomicAdd((unsigned long long*)&st->evals32, nv);
        atomicAdd((unsigned long long*)&st->children, nv);
    }
    if (lane == 0 && n32) {
        atomicAdd((unsigned long long*)&st->evals64, n32);
        atomicAdd((unsigned long long*)&st->mids, n32);
        atomicAdd((unsigned long long*)&st->kept32, n32);
        atomicAdd((unsigned long long*)&st->n32, n32);
    }
    if (!cc) return;
    __shared__ int s_sw[32];
    __shared__ bool s_last;
    if (!arrive_last(&st->cc_done, gridDim.x, &s_last)) return;
    const double gub_new = gb_key_value(__ldcg((const unsigned long long*)&st->gub_new_key));
    const long long S = survivor_list_block(ch, lim, gub_new, true, s_sw);
    if (threadIdx.x == 0) {
        st->cc_done = 0;
        set_survivors(G, st, S);
    }
}

// The same FP32-then-FP64 warp-per-child evaluation over the children of
// many problems in one persistent launch (continuous batching): the work is
// the concatenation of every live problem's children in units of
// GB_BATCH_UNIT; a warp evaluates a unit's children with that problem's
// arguments and then adds its counters and GUB samples to that problem's
// state, exactly as the per-problem kernel does.
#define GB_BATCH_UNIT 4
__global__ void __launch_bounds__(128) k_eval3264_batch(const GbEvalDesc* __restrict__ D, int nreq) {
    __shared__ long long off[GB_BATCH_MAX + 1];
    if (threadIdx.x == 0) {
        long long o = 0;
        for (int q = 0; q < nreq; q++) {
            off[q] = o;
            const GbState* st = D[q].st;
            if (!st->halt) o += (st->nch + GB_BATCH_UNIT - 1) / GB_BATCH_UNIT;
        }
        off[nreq] = o;
    }
    __syncthreads();
    const long long total = off[nreq];
    const int lane = threadIdx.x & 31;
    GB_WSCRATCH_DECL
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long u = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; u < total; u += nw) {
        int lo = 0, hi = nreq - 1;   // the problem q with off[q] <= u < off[q + 1]
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= u) lo = mid;
            else hi = mid - 1;
        }
        const GbEvalDesc& d = D[lo];
        GbState* st = d.st;
        const long long lim = st->nch;
        const double gub_prev = gb_key_value(st->gub_key);
        const long long c0 = (u - off[lo]) * GB_BATCH_UNIT;
        const long long c1 = min(lim, c0 + GB_BATCH_UNIT);
        int red32 = 0, pops32 = 0, red64 = 0, pops64 = 0;
        unsigned long long nv = 0, n32 = 0, key = ~0ull;
        bool has = false;
        for (long long ci = c0; ci < c1; ci++) {
            const int v = eval32_tab_child_w(d.P, d.pool, d.par, d.Tb, d.ch, ci, d.sp, gub_prev, red32, pops32, lane,
                                             ws);
            if (v < 0) continue;
            nv++;
            if (v == 0) continue;
            n32++;
            unsigned long long k2 = ~0ull;
            bool h2 = false;
            eval64_tab_child_w(d.P, d.pool, d.par, d.Tb, d.ch, ci, d.sp, gub_prev, &k2, &h2, red64, pops64, lane, ws);
            if (h2 && k2 < key) key = k2, has = true;
        }
        warp_min_gub(key, has, st);
        warp_add_ops((lane == 0 ? red32 : 0) + pops32, &st->ops32);
        warp_add_ops((lane == 0 ? red64 : 0) + pops64, &st->ops64);
        if (lane == 0 && nv) {
            atomicAdd((unsigned long long*)&st->evals32, nv);
            atomicAdd((unsigned long long*)&st->children, nv);
        }
        if (lane == 0 && n32) {
            atomicAdd((unsigned long long*)&st->evals64, n32);
            atomicAdd((unsigned long long*)&st->mids, n32);
            atomicAdd((unsigned long long*)&st->kept32, n32);
            atomicAdd((unsigned long long*)&st->n32, n32);
        }
    }
}

unsigned grid_for(long long items, int per_block) {
    long long g = (items + per_block - 1) / per_block;
    return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

extern thread_local long long gb_launch_count;   // kernels launched by this thread (gb_kernels.cu)

cudaError_t gb_launch_eval3264_batch(const GbEvalDesc* d_desc, int nreq, long long max_units, cudaStream_t s) {
    if (nreq <= 0) return cudaSuccess;
    if (nreq > GB_BATCH_MAX) return cudaErrorInvalidValue;
    gb_launch_count++;
    const unsigned grid = (unsigned)std::min<long long>(grid_for(max_units * 32, 128), gb_sm_count() * 8);
    k_eval3264_batch<<<grid, 128, 0, s>>>(d_desc, nreq);
    return cudaGetLastError();
}

cudaError_t gb_launch_ptab(const GbProg& P, const GbPool& pool, const GbParents& par, const GbTabs& T,
                           long long K, const GbSplit& sp, GbState* st, cudaStream_t s, const GbEntries* Esel) {
    // row parts of a parent, one per warp, then one block per group tree
    const int parts = ptab_parts(pool), kinds = pool.fp32 ? 3 : 2;
    int row_blocks = (P.max_rows * parts + PTAB_ITEMS - 1) / PTAB_ITEMS;
    if (row_blocks < 1) row_blocks = 1;
    const size_t smem = T.tree_smem ? (size_t)T.max_sum_nodes * sizeof(double2) : 0;
    return gb_launch_ex(k_ptab, dim3((unsigned)(row_blocks + P.n_sum * kinds), (unsigned)K), PTAB_T, smem, s, true, P,
                        pool, par, T, sp, row_blocks, st, Esel ? *Esel : GbEntries{}, Esel ? 1 : 0);
}

cudaError_t gb_launch_eval64_tab(const GbProg& P, const GbPool& pool, const GbParents& par, const GbTabs& T,
                                 const GbChildren& ch, long long Cmax, const GbSplit& sp, bool from_list,
                                 GbState* st, cudaStream_t s) {
    if (T.warp) {
        unsigned g = grid_for(Cmax * 32, 128);
        if (g > gb_sm_count() * 32) g = gb_sm_count() * 32;
        k_eval64_tabw<<<g, 128, 0, s>>>(P, pool, par, T, ch, sp, from_list ? 1 : 0, st);
        return cudaGetLastError();
    }
    unsigned g = grid_for(Cmax, 128);
    if (g > gb_sm_count() * GB_TAB_GRID) g = gb_sm_count() * GB_TAB_GRID;
    return gb_launch_ex(P.outer_sum ? (T.reg ? k_eval64_tab<true, true> : k_eval64_tab<true, false>)
                                    : k_eval64_tab<false, false>,
                        g, 128, 0, s, true, P, pool, par, T, ch, sp, from_list ? 1 : 0, st);
}

cudaError_t gb_launch_ptab_d(const GbProg& P, const GbPool& pool, const GbParents& par, const GbTabs& T,
                             long long K, int B, GbState* st, cudaStream_t s, bool fixed) {
    // threads for the partial-table entries, warps for the segment entries
    const long long items = std::max<long long>((long long)B * P.n_sum << GB_TAB_DBITS,
                                                (long long)P.max_nseg << (GB_TAB_SBITS + 5));
    unsigned g = grid_for(items, 128);
    if (g > (unsigned)gb_sm_count() * 16) g = gb_sm_count() * 16;
    return gb_launch_ex(k_ptab_d, dim3(g, (unsigned)K), 128, 0, s, true, P, pool, par, T, st, fixed ? 1 : 0);
}

cudaError_t gb_launch_child_sums(const GbProg& P, const GbPool& pool, const GbParents& par, const GbTabs& T,
                                 const GbSplit& sp, long long Cmax, int fp32, GbState* st, cudaStream_t s,
                                 bool fixed) {
    if (!T.cs64 || P.n_sum <= 0) return cudaSuccess;
    const int kinds = fp32 ? 3 : 2;
    // fixed: one parent, its 2^flog2 children (the count is not read from the state)
    const long long nch = fixed ? (1LL << sp.flog2) : -1;
    // then, in whole blocks of their own, the first-order verdict tables
    const long long base = (Cmax * P.n_sum * kinds + 127) / 128 * 128;
    const long long mv = T.mv64 ? (Cmax >> sp.flog2) * P.B * (T.mv32 ? 2 : 1) << GB_MV_BITS : 0;
    return gb_launch_ex(k_child_sums, grid_for(base + mv, 128), 128, 0, s, true, P, pool, par, T, sp, Cmax,
                        kinds, st, nch, base);
}

cudaError_t gb_launch_eval3264_tabw(const GbProg& P, const GbPool& pool, const GbParents& par, const GbTabs& T,
                                    const GbChildren& ch, long long Cmax, const GbSplit& sp, GbState* st,
                                    cudaStream_t s, const GbGenConst* cc) {
    unsigned g = grid_for(Cmax * 32, 128);
    if (g > gb_sm_count() * 32) g = gb_sm_count() * 32;
    return gb_launch_ex(k_eval3264_tabw, g, 128, 0, s, true, P, pool, par, T, ch, sp, st, cc ? *cc : GbGenConst{},
                        cc ? 1 : 0);
}

cudaError_t gb_launch_eval32_tab(const GbProg& P, const GbPool& pool, const GbParents& par, const GbTabs& T,
                                 const GbChildren& ch, long long Cmax, const GbSplit& sp, GbState* st,
                                 cudaStream_t s) {
    if (T.warp) {
        unsigned g = grid_for(Cmax * 32, 128);
        if (g > gb_sm_count() * 32) g = gb_sm_count() * 32;
        k_eval32_tabw<<<g, 128, 0, s>>>(P, pool, par, T, ch, sp, st);
        return cudaGetLastError();
    }
    unsigned g = grid_for(Cmax, 128);
    if (g > gb_sm_count() * GB_TAB_GRID) g = gb_sm_count() * GB_TAB_GRID;
    k_eval32_tab<<<g, 128, 0, s>>>(P, pool, par, T, ch, sp, st);
    return cudaGetLastError();
}
