// Helpers shared by the child-evaluation kernels (gb_kernels.cu,
// gb_kernels_tab.cu): the (parent, child index) decomposition of a child,
// its coordinate views, and warp-level reductions into the solver state.
#pragma once
#include "gb_eval.cuh"
#include "gb_launch.h"

namespace gb {

__device__ __forceinline__ double canon_lo(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    if ((b & 0x7fffffffffffffffULL) > 0x7ff0000000000000ULL) return -__longlong_as_double(0x7ff0000000000000LL);
    if ((b << 1) == 0) return 0.0;
    return x;
}

// ---------------------------------------------------------------------------
struct ChildCtx {
    long long p;
    unsigned r, slot;
    int4 info;
    bool valid;
};

__device__ __forceinline__ ChildCtx child_ctx(const GbParents& par, long long ci, const GbSplit& sp) {
    ChildCtx c;
    c.p = ci >> sp.flog2;
    c.r = (unsigned)(ci & ((1LL << sp.flog2) - 1));
    c.info = par.info[c.p];
    c.slot = par.slot[c.p];
    c.valid = c.r < (1u << (c.info.y * sp.mshift));
    return c;
}

// A stored box (no split coordinates) or, with split tables, a child of it.
__device__ __forceinline__ View<double> box_view64(const GbPool& pool, unsigned slot) {
    View<double> v{};
    v.dd = 0;
    v.mshift = 1;
    v.mstride = 2;
    if (pool.recs) {
        v.plo = pool.rlo;
        v.phi = pool.rhi;
        v.rid = pool.rid + (size_t)slot * pool.nb;
        v.B = pool.B;
    } else {
        v.plo = pool.lo64 + (size_t)slot * pool.n;
        v.phi = pool.hi64 + (size_t)slot * pool.n;
    }
    return v;
}
__device__ __forceinline__ View<float> box_view32(const GbPool& pool, unsigned slot) {
    View<float> v{};
    v.dd = 0;
    v.mshift = 1;
    v.mstride = 2;
    if (pool.recs) {
        v.plo = pool.rlo32;
        v.phi = pool.rhi32;
        v.rid = pool.rid + (size_t)slot * pool.nb;
        v.B = pool.B;
    } else {
        v.plo = pool.lo32 + (size_t)slot * pool.n;
        v.phi = pool.hi32 + (size_t)slot * pool.n;
    }
    return v;
}

__device__ __forceinline__ View<double> view64(const GbPool& pool, const GbParents& par, const ChildCtx& c,
                                               const GbSplit& sp) {
    View<double> v = box_view64(pool, c.slot);
    const double* b = par.bnd + (size_t)c.p * sp.dmax * (sp.m + 1);
    v.blo = b;
    v.bhi = b;
    v.c0 = c.info.x;
    v.dd = c.info.y;
    v.mshift = sp.mshift;
    v.mstride = sp.m + 1;
    v.r = c.r;
    return v;
}
__device__ __forceinline__ View<float> view32(const GbPool& pool, const GbParents& par, const ChildCtx& c,
                                              const GbSplit& sp) {
    View<float> v = box_view32(pool, c.slot);
    size_t o = (size_t)c.p * sp.dmax * (sp.m + 1);
    v.blo = par.bnd_rd + o;
    v.bhi = par.bnd_ru + o;
    v.c0 = c.info.x;
    v.dd = c.info.y;
    v.mshift = sp.mshift;
    v.mstride = sp.m + 1;
    v.r = c.r;
    return v;
}

// Cached group sums of a stored box: which 0 = F, 1 = midpoint.
__device__ __forceinline__ CacheRef<double2> cache64(const GbPool& pool, const GbProg& P, unsigned slot, int which) {
    if (pool.recs)
        return CacheRef<double2>{which ? pool.rgmid : pool.rgsum, pool.rid + (size_t)slot * pool.nb, P.gown,
                                 pool.GPB};
    return CacheRef<double2>{(which ? pool.gmid : pool.gsum) + (size_t)slot * pool.NG, nullptr, nullptr, 0};
}
// The box's group sums at diagonal sample j (1 .. S).
__device__ __forceinline__ CacheRef<double2> samp64(const GbPool& pool, const GbProg& P, unsigned slot, int j) {
    if (pool.recs)
        return CacheRef<double2>{pool.rgsamp + (size_t)(j - 1) * pool.R * pool.GPB, pool.rid + (size_t)slot * pool.nb,
                                 P.gown, pool.GPB};
    return CacheRef<double2>{pool.gsamp + ((size_t)slot * pool.S + (j - 1)) * pool.NG, nullptr, nullptr, 0};
}
__device__ __forceinline__ bool has_samp(const GbPool& pool) { return pool.recs ? pool.rgsamp != nullptr : pool.gsamp != nullptr; }

__device__ __forceinline__ CacheRef<float2> cache32(const GbPool& pool, const GbProg& P, unsigned slot) {
    if (pool.recs)
        return CacheRef<float2>{pool.rgsum32, pool.rid + (size_t)slot * pool.nb, P.gown, pool.GPB};
    return CacheRef<float2>{pool.gsum32 + (size_t)slot * pool.NG, nullptr, nullptr, 0};
}

__device__ __forceinline__ void warp_min_gub(unsigned long long key, bool has, GbState* st) {
    unsigned long long k = has ? key : ~0ull;
    for (int o = 16; o; o >>= 1) {
        unsigned long long other = __shfl_down_sync(0xffffffffu, k, o);
        k = other < k ? other : k;
    }
    if ((threadIdx.x & 31) == 0 && k != ~0ull) atomicMin(&st->gub_new_key, k);
}

__device__ __forceinline__ void warp_add_ops(int ops, unsigned long long* dst) {
    unsigned long long v = (unsigned long long)ops;
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, v);
}


// ---- warp-cooperative pieces (one child per warp) ---------------------------
template <typename I> __device__ __forceinline__ I shfl_iv(I v, int src) {
    v.lo = __shfl_sync(0xffffffffu, v.lo, src);
    v.hi = __shfl_sync(0xffffffffu, v.hi, src);
    return v;
}

// Value of dirty group g of sum k for child digits r, NV tables at a time,
// from the group's term-tree segments starting at segment sg (the segments
// of a split position are ordered by sum, group and term, so those of
// (k, g) are the run starting at sg).  The lanes read one segment each
// (load(G, row, v) fills v[0..NV) from the term row or the segment row);
// the values are then pushed in order into the binary counter at each
// segment's level, which forms the group's pairwise tree (Tree::push_level).
// sg advances past the run; nseg = its length.  The counter is kept by lane 0
// alone (its levels are thread-local memory: one copy per warp instead of 32
// identical ones), so `out` is defined in lane 0 only.
template <typename I, int NV, typename L>
__device__ __forceinline__ void warp_group(const GbProg& P, const GbSplitPos& SP, int k, int g, unsigned r,
                                           int& sg, int lane, L load, I* out, int& nseg) {
    Tree<I> tr[NV];
    for (int t = 0; t < NV; t++) tr[t].init();
    nseg = 0;
    const int send = SP.seg0 + SP.nseg;
    for (;;) {
        const int i = sg + lane;
        bool mem = false;
        int lev = 0;
        I v[NV];
        for (int t = 0; t < NV; t++) v[t].lo = v[t].hi = 0;
        if (i < send) {
            const GbSeg G = P.segs[i];
            mem = G.sum == k && G.group == g;
            if (mem) {
                lev = G.level;
                load(G, G.base + (int)((r >> G.shift) & G.mask), v);
            }
        }
        const int rr = __popc(__ballot_sync(0xffffffffu, mem));
        if (rr == 0) break;
        for (int j = 0; j < rr; j++) {
            const int lj = __shfl_sync(0xffffffffu, lev, j);
            for (int t = 0; t < NV; t++) {
                const I x = shfl_iv(v[t], j);
                if (lane == 0) tr[t].push_level(x, lj);   // the counter lives in lane 0 only
            }
        }
        nseg += rr;
        sg += rr;
        if (rr < 32) break;
    }
    if (lane == 0)
        for (int t = 0; t < NV; t++) out[t] = tr[t].result();
}

// A block's arrival at a grid-wide counter of n blocks; every thread calls
// it and gets true in the last block to arrive.  The block's writes before
// the call (any thread's: the barrier orders them before thread 0's release
// fence, which is cumulative) are visible to that last block after it (its
// thread 0 acquires before the second barrier).  Fences at GPU scope with
// acquire-release strength: the ordering this needs, without the cost of a
// sequentially consistent fence in every thread.
__device__ __forceinline__ bool arrive_last(unsigned* counter, unsigned n, bool* s_flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        const bool last = atomicAdd(counter, 1u) == n - 1;
        if (last) asm volatile("fence.acq_rel.gpu;" ::: "memory");
        *s_flag = last;
    }
    __syncthreads();
    return *s_flag;
}

// Exclusive scan of one int per thread over a block (any multiple of 32
// threads up to 1024; sw: 32 ints of shared memory); *total gets the sum.
__device__ __forceinline__ int block_excl_scan(int v, int* sw, int* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) sw[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = lane < nw ? sw[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) sw[lane] = t;
    }
    __syncthreads();
    *total = sw[nw - 1];
    return x - v + (w ? sw[w - 1] : 0);
}

// The survivors of a generation (children kept by the FP64 tests whose lower
// bound is not above the new incumbent), in ascending order, listed by one
// block: each thread takes a contiguous run of at most 64 children (n <= 64
// blockDim.x), loads its flags and bounds eight at a time (independent
// loads), keeps the verdicts as a bit mask, and one block scan places the
// runs.  `cg`: the flags were written by other blocks of the running kernel
// and are read through L2.  Returns the count (every thread).
__device__ __forceinline__ long long survivor_list_block(const GbChildren& ch, long long n, double gub_new, bool cg,
                                                         int* sw) {
    const int per = (int)((n + blockDim.x - 1) / blockDim.x);
    const long long i0 = (long long)threadIdx.x * per;
    unsigned long long m = 0;
    for (int c0 = 0; c0 < per; c0 += 8) {
        unsigned char f[8];
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const long long i = i0 + c0 + u;
            const bool in = c0 + u < per && i < n;
            f[u] = in ? (cg ? __ldcg(ch.flag + i) : ch.flag[i]) : (unsigned char)0;
            v[u] = in ? (cg ? __ldcg(ch.flo + i) : ch.flo[i]) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; u++)
            if (f[u] != 0 && !(v[u] > gub_new)) m |= 1ull << (c0 + u);
    }
    int tot;
    long long o = block_excl_scan(__popcll(m), sw, &tot);
    while (m) {
        const int b = __ffsll((long long)m) - 1;
        ch.surv[o++] = (unsigned)(i0 + b);
        m &= m - 1;
    }
    return tot;
}

// The generation's survivor count and what it implies: overflow when the
// pool cannot take them or their block records do not fit (after the
// generation's record collection, if it ran).
__device__ __forceinline__ void set_survivors(const GbGenConst& G, GbState* st, long long S) {
    st->kept = S;
    const long long room = st->nfree + (st->cap - st->bump);
    st->overflow = (S > room || (G.nrec && S * G.nrec > st->rec_nfree + (G.R - st->rec_bump))) ? 1 : 0;
}

}  // namespace gb
