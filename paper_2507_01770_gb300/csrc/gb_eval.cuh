// Device evaluation of the compiled objective over one box (one thread).
//
//  * natural interval extension of f (section 2.1): the template bytecode of
//    every sum and the outer bytecode are interpreted instruction by
//    instruction with the outward-rounded operations of gb_interval.cuh;
//  * sums are reduced in a fixed order: within a group of terms by a pairwise
//    tree in term order, then over the groups by a pairwise tree in group
//    order.  The tree is computed with a binary counter (level L holds the
//    sum of 2^L consecutive items), which forms exactly the in-place pairwise
//    tree a[i] += a[i + s], s = 1, 2, 4, ...;
//  * a child of a cached parent recomputes only the groups that touch its
//    split block and reuses the parent's cached group sums for the rest;
//  * the interval partials of the active block's coordinates (the DLB/DUB of
//    the first-order test, section 3.1) come from a reverse sweep over the
//    outer bytecode and, per term, over the template bytecode seeded with
//    [1, 1]; leaf adjoints are accumulated per coordinate in ascending term
//    and leaf order, then multiplied by the sum's outer adjoint.
#pragma once
#include "gb_internal.h"
#include "gb_interval.cuh"

namespace gb {

template <typename T> struct Prec;
template <> struct Prec<double> {
    typedef iv64 I;
    static __device__ __forceinline__ I coef(const GbProg& P, int t, int idx) {
        double c = __ldg(P.tab64[t] + idx);
        return I{c, c};
    }
    static __device__ __forceinline__ I cst(const GbIns& in) { return I{in.c, in.c}; }
};
template <> struct Prec<float> {
    typedef iv32 I;
    static __device__ __forceinline__ I coef(const GbProg& P, int t, int idx) {
        float2 c = __ldg(P.tab32[t] + idx);
        return I{c.x, c.y};
    }
    static __device__ __forceinline__ I cst(const GbIns& in) { return I{in.clo32, in.chi32}; }
};

// Coordinates of a box in precision T.  Coordinates [c0, c0 + dd) come from
// a split table: piece `digit` of coordinate c0 + k spans
// [blo[k * (m + 1) + digit], bhi[k * (m + 1) + digit + 1]]; the others from
// the row (plo, phi).  dd = 0 views a plain box.
template <typename T> struct View {
    const T* plo;
    const T* phi;
    const T* blo;
    const T* bhi;
    int c0, dd, mshift, mstride;
    unsigned r;
    // block records: plo/phi are the record stores and rid the box's record
    // ids (coordinate j in record rid[j / B] at j % B); null for a dense row
    const unsigned* rid = nullptr;
    int B = 1;
    __device__ __forceinline__ typename Prec<T>::I get(int j) const {
        unsigned k = (unsigned)(j - c0);
        typename Prec<T>::I x;
        if (k < (unsigned)dd) {
            int dig = (r >> (k * mshift)) & ((1 << mshift) - 1);
            x.lo = blo[k * mstride + dig];
            x.hi = bhi[k * mstride + dig + 1];
        } else if (rid) {
            const int b = j / B;
            const size_t o = (size_t)rid[b] * B + (j - b * B);
            x.lo = plo[o];
            x.hi = phi[o];
        } else {
            x.lo = plo[j];
            x.hi = phi[j];
        }
        return x;
    }
};

// Cached group sums of one box: a dense row (rid == null) or the box's block
// records (group g in record rid[gown[g].x] at index gown[g].y).
template <typename C> struct CacheRef {
    const C* base;
    const unsigned* rid;
    const int2* gown;
    int GPB;
    __device__ __forceinline__ C operator[](int g) const {
        if (rid) {
            const int2 o = gown[g];
            return base[(size_t)rid[o.x] * GPB + o.y];
        }
        return base[g];
    }
};

// The FP64 midpoint sample point m = RN(0.5 lo + 0.5 hi) of each coordinate.
struct MidView {
    View<double> v;
    __device__ __forceinline__ iv64 get(int j) const {
        iv64 x = v.get(j);
        double m = __dadd_rn(__dmul_rn(0.5, x.lo), __dmul_rn(0.5, x.hi));
        return iv64{m, m};
    }
};

// Diagonal sample point j of S: coordinate i is boundary j of the (S + 1)-piece
// partition of [lo_i, hi_i], RN(lo + RN(RN(RN(hi - lo) / (S + 1)) * j)) (the
// split-boundary rounding), j in 1 .. S.
struct SampleView {
    View<double> v;
    int j, m1;
    __device__ __forceinline__ iv64 get(int i) const {
        const iv64 x = v.get(i);
        const double w = __dsub_rn(x.hi, x.lo);
        const double q = __ddiv_rn(w, (double)m1);
        const double s = __dmul_rn(q, (double)j);
        const double p = __dadd_rn(x.lo, s);
        return iv64{p, p};
    }
};

// Binary-counter pairwise tree.
template <typename I, bool PROD = false> struct Tree {
    I lvl[20];
    unsigned cnt;
    // the tree's operation: sums (ISUM) or products (IPROD)
    __device__ __forceinline__ static I comb(I a, I b) {
        if constexpr (PROD) return imul(a, b);
        else return iadd(a, b);
    }
    __device__ __forceinline__ void init() { cnt = 0; }
    __device__ __forceinline__ void push(I v) {
        unsigned c = cnt;
        int L = 0;
        while (c & 1u) {
            v = comb(lvl[L], v);
            c >>= 1;
            L++;
        }
        lvl[L] = v;
        cnt++;
    }
    // Push the sum of an aligned block of 2^L items (cnt a multiple of 2^L):
    // the same levels as pushing the block's items one by one, when v is
    // the block's own in-place pairwise sum.
    __device__ __forceinline__ void push_level(I v, int L) {
        unsigned c = cnt >> L;
        int lev = L;
        while (c & 1u) {
            v = comb(lvl[lev], v);
            c >>= 1;
            lev++;
        }
        lvl[lev] = v;
        cnt += 1u << L;
    }
    __device__ __forceinline__ I result() const {
        I r;
        if (!cnt) { r.lo = PROD ? 1 : 0; r.hi = PROD ? 1 : 0; return r; }
        // levels present in ascending order (the set bits of cnt)
        unsigned c = cnt;
        r = lvl[__ffs(c) - 1];
        for (c &= c - 1; c; c &= c - 1) r = comb(lvl[__ffs(c) - 1], r);
        return r;
    }
};

// Division, square root and the transcendentals, kept out of line: the
// interpreter loops below stay small in the instruction cache, and these
// operations cost far more than a call.
template <typename I> __device__ __noinline__ I slow_fwd(int op, I a, I b) {
    switch (op) {
    case D_DIV: return idiv(a, b);
    case D_SQRT: return isqrt(a);
    case D_EXP: return iexp(a);
    case D_SIN: return itrig(a, false);
    case D_STEP: return istep(a);
    default: return itrig(a, true);   // D_COS
    }
}
// Adjoint contributions of node v = op(a, b) with adjoint g: *da to operand
// a (and *db to b for a division).
template <typename I> __device__ __noinline__ void slow_rev(int op, I g, I va, I vb, I vt, I* da, I* db) {
    typedef decltype(g.lo) T;
    switch (op) {
    case D_DIV: {
        I rb = ircp(vb);
        *da = imul(g, rb);
        *db = imul(g, ineg(imul(vt, rb)));
        break;
    }
    case D_SQRT: *da = imul(g, iscale(ircp(vt), (T)0.5)); break;
    case D_SIN: *da = imul(g, itrig(va, true)); break;
    case D_STEP: {   // H' = 0 off the jump; unbounded on a box that holds it (nonzero adjoint)
        const bool jump = !(va.lo >= (T)0) && !(va.hi < (T)0);
        const bool live = !(g.lo == (T)0 && g.hi == (T)0);
        const T inf = (T)INFINITY;
        da->lo = jump && live ? -inf : (T)0;
        da->hi = jump && live ? inf : (T)0;
        break;
    }
    default: *da = imul(g, ineg(itrig(va, false))); break;   // D_COS
    }
}

// The same, for lanes 0 and 1 of a warp interpreting the same template
// together (PAIR interpreters): exp, sin and cos evaluate their two
// endpoints in the two lanes (iexp_pair, itrig_pair); the other operations
// run in both lanes alike.
template <typename I> __device__ __noinline__ I slow_fwd_pair(int op, I a, I b) {
    switch (op) {
    case D_EXP: return iexp_pair(a);
    case D_SIN: return itrig_pair(a, false);
    case D_COS: return itrig_pair(a, true);
    default: return slow_fwd(op, a, b);
    }
}
template <typename I> __device__ __noinline__ void slow_rev_pair(int op, I g, I va, I vb, I vt, I* da, I* db) {
    switch (op) {
    case D_SIN: *da = imul(g, itrig_pair(va, true)); break;
    case D_COS: *da = imul(g, ineg(itrig_pair(va, false))); break;
    default: slow_rev(op, g, va, vb, vt, da, db); break;
    }
}

// Forward interpretation of one template for term index i; returns the root.
// `sins` / `pre` (both or neither): the template's instructions and the
// values of its coordinate and coefficient loads, staged by stage_term.
// PAIR: run by lanes 0 and 1 of a warp together (slow_fwd_pair).
template <typename T, typename V, bool PAIR = false>
__device__ __forceinline__ typename Prec<T>::I term_fwd(const GbProg& P, const GbSum& S, int i,
                                                         const V& X, typename Prec<T>::I* R, int& ops,
                                                         const GbIns* sins = nullptr,
                                                         const typename Prec<T>::I* pre = nullptr) {
    typedef typename Prec<T>::I I;
    const GbIns* ins = sins ? sins : P.tins + S.ins0;
    for (int t = 0; t < S.nins; t++) {
        GbIns in = ins[t];
        ops += in.pad & 0xff;
        I v;
        switch (in.op) {
        case D_CONST: v = Prec<T>::cst(in); break;
        case D_PI: v = pi_iv((T)0); break;
        case D_EULER: v = e_iv((T)0); break;
        case D_IVAR: v = pre ? pre[t] : X.get(i + in.aux); break;
        case D_COEF: v = pre ? pre[t] : Prec<T>::coef(P, in.aux, i + in.aux2); break;
        case D_ADD: v = iadd(R[in.a], R[in.b]); break;
        case D_SUB: v = isub(R[in.a], R[in.b]); break;
        case D_MUL: v = imul(R[in.a], R[in.b]); break;
        case D_NEG: v = ineg(R[in.a]); break;
        case D_SQR: v = isqr(R[in.a]); break;
        case D_DIV: v = slow_fwd(in.op, R[in.a], R[in.b]); break;
        case D_SQRT:
        case D_STEP: v = slow_fwd(in.op, R[in.a], R[in.a]); break;
        case D_EXP:
        case D_SIN:
        case D_COS: v = PAIR ? slow_fwd_pair(in.op, R[in.a], R[in.a]) : slow_fwd(in.op, R[in.a], R[in.a]); break;
        case D_SCALE:
            if (in.clo32 == in.chi32 || sizeof(T) == 8)
                v = iscale(R[in.a], sizeof(T) == 8 ? (T)in.c : (T)in.clo32);
            else
                v = imul(R[in.a], mk<T>((T)in.clo32, (T)in.chi32));
            break;
        default: v.lo = 0; v.hi = 0; break;
        }
        R[t] = v;
    }
    return R[S.nins - 1];
}

// Warp-cooperative staging for term_fwd: lane t (t < nins) loads instruction
// t of the template into `sins` and, for a coordinate or coefficient load,
// its value into `pre` -- the loads of all instructions in flight at once,
// instead of one after the other in the interpreter loop.  Every lane of the
// warp calls it (the views are the same in every lane).
template <typename T, typename V>
__device__ __forceinline__ void stage_term(const GbProg& P, const GbSum& S, int i, const V& X, GbIns* sins,
                                           typename Prec<T>::I* pre, int lane) {
    if (lane < S.nins) {
        const GbIns in = P.tins[S.ins0 + lane];
        sins[lane] = in;
        if (in.op == D_IVAR) pre[lane] = X.get(i + in.aux);
        else if (in.op == D_COEF) pre[lane] = Prec<T>::coef(P, in.aux, i + in.aux2);
    }
    __syncwarp();
}

// Reverse sweep over a bytecode list (forward values V, adjoints A already
// seeded).  Node t pushes into its first, then its second operand; a node's
// adjoint thus receives its consumers' contributions in descending order.
template <typename T, bool PAIR = false>
__device__ __forceinline__ void reverse_sweep(const GbIns* ins, int nins, const typename Prec<T>::I* V,
                                              typename Prec<T>::I* A, int& ops) {
    typedef typename Prec<T>::I I;
    for (int t = nins - 1; t >= 0; t--) {
        GbIns in = ins[t];
        ops += (in.pad >> 8) & 0xff;
        I g = A[t];
        switch (in.op) {
        case D_ADD:
            A[in.a] = iadd(A[in.a], g);
            A[in.b] = iadd(A[in.b], g);
            break;
        case D_SUB:
            A[in.a] = iadd(A[in.a], g);
            A[in.b] = iadd(A[in.b], ineg(g));
            break;
        case D_MUL: {
            I va = V[in.a], vb = V[in.b];
            A[in.a] = iadd(A[in.a], imul(g, vb));
            A[in.b] = iadd(A[in.b], imul(g, va));
            break;
        }
        case D_DIV: {
            I da, db;
            slow_rev(in.op, g, V[in.a], V[in.b], V[t], &da, &db);
            A[in.a] = iadd(A[in.a], da);
            A[in.b] = iadd(A[in.b], db);
            break;
        }
        case D_NEG: A[in.a] = iadd(A[in.a], ineg(g)); break;
        case D_SQR: A[in.a] = iadd(A[in.a], imul(g, iscale(V[in.a], (T)2))); break;
        case D_EXP: A[in.a] = iadd(A[in.a], imul(g, V[t])); break;
        case D_SQRT:
        case D_SIN:
        case D_STEP:
        case D_COS: {
            I da, db;
            if (PAIR) slow_rev_pair(in.op, g, V[in.a], V[in.a], V[t], &da, &db);
            else slow_rev(in.op, g, V[in.a], V[in.a], V[t], &da, &db);
            A[in.a] = iadd(A[in.a], da);
            break;
        }
        case D_SCALE:
            if (in.clo32 == in.chi32 || sizeof(T) == 8)
                A[in.a] = iadd(A[in.a], iscale(g, sizeof(T) == 8 ? (T)in.c : (T)in.clo32));
            else
                A[in.a] = iadd(A[in.a], imul(g, mk<T>((T)in.clo32, (T)in.chi32)));
            break;
        default: break;
        }
    }
}

// Sum (IPROD: product) of the terms of one group (local group g of sum S).
template <bool PROD, typename T, typename V>
__device__ __forceinline__ typename Prec<T>::I group_reduce(const GbProg& P, const GbSum& S, int g, const V& X,
                                                             typename Prec<T>::I* R, int& ops) {
    typedef typename Prec<T>::I I;
    GbGroup G = P.groups[S.group0 + g];
    Tree<I, PROD> tr;
    tr.init();
    for (int t = 0; t < G.count; t++) tr.push(term_fwd<T>(P, S, S.first + (G.t0 + t) * S.step, X, R, ops));
    ops += (PROD ? 8 : 2) * (G.count > 0 ? G.count - 1 : 0);
    return tr.result();
}

// PR: the program may hold IPROD reductions (kernels are instantiated for
// both, so sum-only programs carry no product code).
template <bool PR, typename T, typename V>
__device__ __forceinline__ typename Prec<T>::I group_sum(const GbProg& P, const GbSum& S, int g, const V& X,
                                                          typename Prec<T>::I* R, int& ops) {
    if constexpr (PR) {
        if (S.prod) return group_reduce<true, T>(P, S, g, X, R, ops);
    }
    return group_reduce<false, T>(P, S, g, X, R, ops);
}

// Value of product k: the groups dirty for block blk recomputed, the others
// from `cache` (NULL: all recomputed), reduced by the product tree.
template <typename T, typename V, typename C>
__device__ __noinline__ typename Prec<T>::I prod_value(const GbProg& P, int k, int blk, const V& X,
                                                        const CacheRef<C>* cache, typename Prec<T>::I* R,
                                                        int& ops) {
    typedef typename Prec<T>::I I;
    const GbSum S = P.sums[k];
    const int2 dr = cache ? (blk >= 0 ? P.dirty[blk * P.n_sum + k] : make_int2(0, 0)) : make_int2(0, S.ngroups);
    Tree<I, true> tr;
    tr.init();
    for (int g = 0; g < S.ngroups; g++) {
        I v;
        if (g >= dr.x && g < dr.y) {
            v = group_reduce<true, T>(P, S, g, X, R, ops);
        } else {
            C c = (*cache)[S.group0 + g];
            v.lo = c.x;
            v.hi = c.y;
        }
        tr.push(v);
    }
    ops += 8 * (S.ngroups > 0 ? S.ngroups - 1 : 0);
    return tr.result();
}

// Value of every sum: dirty groups recomputed, the others read from `cache`
// (one interval per global group; NULL: recompute everything).
template <bool PR, typename T, typename V, typename C>
__device__ __forceinline__ void sum_values(const GbProg& P, int blk, const V& X, const CacheRef<C>* cache,
                                           typename Prec<T>::I* R, typename Prec<T>::I* sums, int& ops) {
    typedef typename Prec<T>::I I;
    for (int k = 0; k < P.n_sum; k++) {
        GbSum S = P.sums[k];
        // with a cache: the dirty groups of block blk recomputed (blk < 0: none)
        if constexpr (PR) {
            if (S.prod) {
                sums[k] = prod_value<T>(P, k, blk, X, cache, R, ops);
                continue;
            }
        }
        int2 dr = cache ? (blk >= 0 ? P.dirty[blk * P.n_sum + k] : make_int2(0, 0)) : make_int2(0, S.ngroups);
        Tree<I> tr;
        tr.init();
        for (int g = 0; g < S.ngroups; g++) {
            I v;
            if (g >= dr.x && g < dr.y) {
                v = group_reduce<false, T>(P, S, g, X, R, ops);
            } else {
                C c = (*cache)[S.group0 + g];
                v.lo = c.x;
                v.hi = c.y;
            }
            tr.push(v);
        }
        ops += 2 * (S.ngroups > 0 ? S.ngroups - 1 : 0);
        sums[k] = tr.result();
    }
}

// ---- IPROD adjoints ----
// Adjoint of item q of the pairwise product tree over m items (the tree of
// Tree<I, true>) when the product has adjoint a: reverse mode over the
// tree's products, where every node feeds one product, so each level
// multiplies the adjoint by the value of the node's partner (the product of
// a run of items), taken from the top level down.  get(i) gives item i.
template <typename I, typename G>
__device__ __forceinline__ I tree_item_adjoint(I a, int m, int q, const G& get, int& ops) {
    int plo[20], phi[20], np = 0;
    int h = q;   // q's node at level s starts at item h (a multiple of s)
    for (int s = 1; s < m; s <<= 1) {
        if ((h & (2 * s - 1)) == 0) {   // left operand: partner [h + s, h + 2s) if present
            if (h + s < m) plo[np] = h + s, phi[np] = min(h + 2 * s, m), np++;
        } else {                        // right operand of the node at h - s
            plo[np] = h - s, phi[np] = h, np++;
            h -= s;
        }
    }
    for (int t = np - 1; t >= 0; t--) {
        Tree<I, true> tr;
        tr.init();
        for (int i = plo[t]; i < phi[t]; i++) tr.push(get(i));
        ops += 8 * (phi[t] - plo[t]);
        a = imul(a, tr.result());
    }
    return a;
}

// The adjoint, within product S (seed [1, 1] at the product), of its term
// with ordinal tt: through the tree over the groups, then through the
// group's own tree.  Group values: from `cache` except the groups dirty for
// block dblk (all recomputed without a cache).
template <typename T, typename V, typename C>
__device__ __noinline__ typename Prec<T>::I prod_term_seed(const GbProg& P, int ks, int tt, const V& X,
                                                            const CacheRef<C>* cache, int dblk,
                                                            typename Prec<T>::I* R, int& ops) {
    typedef typename Prec<T>::I I;
    const GbSum S = P.sums[ks];
    int gl = 0;
    while (gl + 1 < S.ngroups && P.groups[S.group0 + gl + 1].t0 <= tt) gl++;
    const GbGroup G = P.groups[S.group0 + gl];
    const int2 dr = cache ? (dblk >= 0 ? P.dirty[dblk * P.n_sum + ks] : make_int2(0, 0)) : make_int2(0, S.ngroups);
    auto gval = [&](int g) {
        I v;
        if (g >= dr.x && g < dr.y) {
            v = group_reduce<true, T>(P, S, g, X, R, ops);
        } else {
            C c = (*cache)[S.group0 + g];
            v.lo = c.x;
            v.hi = c.y;
        }
        return v;
    };
    auto tval = [&](int t) { return term_fwd<T>(P, S, S.first + (G.t0 + t) * S.step, X, R, ops); };
    I a = mk<T>((T)1, (T)1);
    a = tree_item_adjoint(a, S.ngroups, gl, gval, ops);
    return tree_item_adjoint(a, G.count, tt - G.t0, tval, ops);
}

// Outer forward pass; O receives all outer registers, returns F.
template <typename T, typename V>
__device__ __forceinline__ typename Prec<T>::I outer_fwd(const GbProg& P, const V& X,
                                                          const typename Prec<T>::I* sums,
                                                          typename Prec<T>::I* O, int& ops) {
    typedef typename Prec<T>::I I;
    for (int t = 0; t < P.n_outer; t++) {
        GbIns in = P.outer[t];
        ops += in.pad & 0xff;
        I v;
        switch (in.op) {
        case D_CONST: v = Prec<T>::cst(in); break;
        case D_PI: v = pi_iv((T)0); break;
        case D_EULER: v = e_iv((T)0); break;
        case D_VAR: v = X.get(in.aux); break;
        case D_ISUMV: v = sums[in.aux]; break;
        case D_ADD: v = iadd(O[in.a], O[in.b]); break;
        case D_SUB: v = isub(O[in.a], O[in.b]); break;
        case D_MUL: v = imul(O[in.a], O[in.b]); break;
        case D_NEG: v = ineg(O[in.a]); break;
        case D_SQR: v = isqr(O[in.a]); break;
        case D_DIV:
        case D_SQRT:
        case D_EXP:
        case D_SIN:
        case D_STEP:
        case D_COS: v = slow_fwd(in.op, O[in.a], O[in.b]); break;
        case D_SCALE:
            if (in.clo32 == in.chi32 || sizeof(T) == 8)
                v = iscale(O[in.a], sizeof(T) == 8 ? (T)in.c : (T)in.clo32);
            else
                v = imul(O[in.a], mk<T>((T)in.clo32, (T)in.chi32));
            break;
        default: v.lo = 0; v.hi = 0; break;
        }
        O[t] = v;
    }
    return O[P.outer_root];
}

// First-order test over the coordinates of block blk (section 3.1): returns
// true if some partial excludes 0 with the corresponding face off the domain
// edge.  X64 gives the FP64 box for the edge comparison.  G (optional)
// receives the partials of the block.  Needs the outer registers O of the
// forward pass.  A product's term templates are seeded with the term's
// adjoint in the product (prod_term_seed; group values from gcache except
// the groups dirty for block dblk, all recomputed when gcache is null).
template <bool PR, typename T, typename V, typename C>
__device__ __forceinline__ bool block_mono(const GbProg& P, int blk, const V& X, const View<double>& X64,
                                           const typename Prec<T>::I* O, typename Prec<T>::I* OA,
                                           typename Prec<T>::I* R, typename Prec<T>::I* RA,
                                           double* Gout, const CacheRef<C>* gcache, int dblk, int& ops) {
    typedef typename Prec<T>::I I;
    // outer adjoints
    for (int t = 0; t < P.n_outer; t++) OA[t] = mk<T>((T)0, (T)0);
    OA[P.outer_root] = mk<T>((T)1, (T)1);
    reverse_sweep<T>(P.outer, P.n_outer, O, OA, ops);

    const int c0 = blk * P.B;
    const int c1 = min(P.n, c0 + P.B);
    I W[GB_MAX_ISUM][GB_MAX_WIN];
    unsigned touched[GB_MAX_ISUM];
    int cur[GB_MAX_ISUM];
    for (int k = 0; k < P.n_sum; k++) {
        GbSum S = P.sums[k];
        // first term whose touched range reaches c0
        int need = c0 - S.off_max - S.first;
        cur[k] = need <= 0 ? 0 : (need + S.step - 1) / S.step;
        touched[k] = 0;
        for (int w = 0; w < GB_MAX_WIN; w++) W[k][w] = mk<T>((T)0, (T)0);
    }
    bool mono = false;
    for (int j = c0; j < c1; j++) {
        I g = mk<T>((T)0, (T)0);
        for (int v = 0; v < P.n_var_leaves; v++) {
            GbVarLeaf L = P.var_leaves[v];
            if (L.coord == j) g = iadd(g, OA[L.reg]), ops += 2;
        }
        for (int k = 0; k < P.n_sum; k++) {
            GbSum S = P.sums[k];
            if (!S.has_var) continue;
            while (cur[k] < S.count && S.first + cur[k] * S.step + S.off_min <= j) {
                int i = S.first + cur[k] * S.step;
                I seed = mk<T>((T)1, (T)1);
                if constexpr (PR) {
                    if (S.prod) seed = prod_term_seed<T>(P, k, cur[k], X, gcache, dblk, R, ops);
                }
                term_fwd<T>(P, S, i, X, R, ops);
                for (int t = 0; t < S.nins; t++) RA[t] = mk<T>((T)0, (T)0);
                RA[S.nins - 1] = seed;
                const GbIns* ins = P.tins + S.ins0;
                reverse_sweep<T>(ins, S.nins, R, RA, ops);
                for (int t = 0; t < S.nins; t++) {
                    GbIns in = ins[t];
                    if (in.op != D_IVAR) continue;
                    int cc = i + in.aux;
                    if (cc < c0 || cc >= c1) continue;
                    int w = cc & (GB_MAX_WIN - 1);
                    W[k][w] = iadd(W[k][w], RA[t]);
                    ops += 2;
                    touched[k] |= 1u << w;
                }
                cur[k]++;
            }
            int w = j & (GB_MAX_WIN - 1);
            if (touched[k] & (1u << w)) {
                g = iadd(g, imul(OA[S.outer_reg], W[k][w]));
                ops += 4;
                W[k][w] = mk<T>((T)0, (T)0);
                touched[k] &= ~(1u << w);
            }
        }
        if (Gout) {
            Gout[2 * (j - c0)] = (double)g.lo;
            Gout[2 * (j - c0) + 1] = (double)g.hi;
        }
        iv64 x = X64.get(j);
        if ((gt_zero(g.lo) && !same_value(x.lo, __ldg(P.l + j))) ||
            (lt_zero(g.hi) && !same_value(x.hi, __ldg(P.u + j)))) {
            mono = true;
            if (!Gout) break;
        }
    }
    return mono;
}

// ---- cached coordinate partials (first-order test on every coordinate) ----
// D_kj: the sum over the terms of sum k of their leaf adjoints for
// coordinate j, accumulated from [0, 0] in ascending term and leaf order
// (the value block_mono multiplies by the sum's outer adjoint); stored as
// row[k * stride + (j - j0)] (a dense row: stride n, j0 0; a block record:
// stride B, j0 its first coordinate), an untouched pair as (+inf, -inf).
__device__ __forceinline__ bool d_touched(double2 d) {
    return !(__double_as_longlong(d.x) == 0x7ff0000000000000LL &&
             __double_as_longlong(d.y) == (long long)0xfff0000000000000ULL);
}

// D of the coordinates of block blk over box X into row (FP64).
template <typename V>
__device__ __noinline__ void block_D(const GbProg& P, int blk, const V& X, iv64* R, iv64* RA, double2* row,
                                        int stride, int j0, int& ops) {
    const int c0 = blk * P.B;
    const int c1 = min(P.n, c0 + P.B);
    iv64 W[GB_MAX_ISUM][GB_MAX_WIN];
    unsigned touched[GB_MAX_ISUM];
    int cur[GB_MAX_ISUM];
    for (int k = 0; k < P.n_sum; k++) {
        GbSum S = P.sums[k];
        int need = c0 - S.off_max - S.first;
        cur[k] = need <= 0 ? 0 : (need + S.step - 1) / S.step;
        touched[k] = 0;
        for (int w = 0; w < GB_MAX_WIN; w++) W[k][w] = iv64{0.0, 0.0};
    }
    for (int j = c0; j < c1; j++) {
        for (int k = 0; k < P.n_sum; k++) {
            GbSum S = P.sums[k];
            double2 out = make_double2(__longlong_as_double(0x7ff0000000000000LL),
                                       __longlong_as_double((long long)0xfff0000000000000ULL));
            if (S.has_var) {
                while (cur[k] < S.count && S.first + cur[k] * S.step + S.off_min <= j) {
                    int i = S.first + cur[k] * S.step;
                    term_fwd<double>(P, S, i, X, R, ops);
                    for (int t = 0; t < S.nins; t++) RA[t] = iv64{0.0, 0.0};
                    RA[S.nins - 1] = iv64{1.0, 1.0};
                    const GbIns* ins = P.tins + S.ins0;
                    reverse_sweep<double>(ins, S.nins, R, RA, ops);
                    for (int t = 0; t < S.nins; t++) {
                        GbIns in = ins[t];
                        if (in.op != D_IVAR) continue;
                        int cc = i + in.aux;
                        if (cc < c0 || cc >= c1) continue;
                        int w = cc & (GB_MAX_WIN - 1);
                        W[k][w] = iadd(W[k][w], RA[t]);
                        ops += 2;
                        touched[k] |= 1u << w;
                    }
                    cur[k]++;
                }
                int w = j & (GB_MAX_WIN - 1);
                if (touched[k] & (1u << w)) {
                    out = make_double2(W[k][w].lo, W[k][w].hi);
                    W[k][w] = iv64{0.0, 0.0};
                    touched[k] &= ~(1u << w);
                }
            }
            row[(size_t)k * stride + (j - j0)] = out;
        }
    }
}

// Blocks whose D a split of block blk changes: the blocks with a coordinate
// within the widest term's reach (its IDX_VAR offset range) of the block.
__device__ __forceinline__ int2 d_affected(const GbProg& P, int blk) {
    int tw = 0;
    for (int k = 0; k < P.n_sum; k++)
        if (P.sums[k].has_var) tw = max(tw, P.sums[k].off_max - P.sums[k].off_min);
    const int c0 = blk * P.B, c1 = min(P.n, c0 + P.B) - 1;
    return make_int2(max(0, c0 - tw) / P.B, min(P.nb - 1, (c1 + tw) / P.B));
}

// First-order test of block blk from cached D and the box's own outer
// adjoints OA (the operations of block_mono after its term sweeps).
__device__ __forceinline__ bool cached_mono(const GbProg& P, int blk, const View<double>& X64, const iv64* OA,
                                            const double2* row, int stride, int j0, int& ops) {
    const int c0 = blk * P.B;
    const int c1 = min(P.n, c0 + P.B);
    for (int j = c0; j < c1; j++) {
        iv64 g{0.0, 0.0};
        for (int v = 0; v < P.n_var_leaves; v++) {
            GbVarLeaf L = P.var_leaves[v];
            if (L.coord == j) g = iadd(g, OA[L.reg]), ops += 2;
        }
        for (int k = 0; k < P.n_sum; k++) {
            const GbSum S = P.sums[k];
            if (!S.has_var) continue;
            const double2 d = row[(size_t)k * stride + (j - j0)];
            if (!d_touched(d)) continue;
            g = iadd(g, imul(OA[S.outer_reg], iv64{d.x, d.y}));
            ops += 4;
        }
        iv64 x = X64.get(j);
        if ((gt_zero(g.lo) && !same_value(x.lo, __ldg(P.l + j))) ||
            (lt_zero(g.hi) && !same_value(x.hi, __ldg(P.u + j))))
            return true;
    }
    return false;
}

}  // namespace gb
