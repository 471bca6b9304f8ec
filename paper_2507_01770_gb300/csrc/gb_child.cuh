// Helpers shared by the child-evaluation kernels (gb_kernels.cu,
// gb_kernels_tab.cu): the (parent, child index) decomposition of a child,
// its coordinate views, and warp-level reductions into the solver state.
#pragma once
#include "gb_eval.cuh"
#include "gb_launch.h"

namespace gb {

__device__ __forceinline__ double canon_lo(double x) {
    if (x != x) return -__longlong_as_double(0x7ff0000000000000LL);
    if (x == 0.0) return 0.0;
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

__device__ __forceinline__ View<double> view64(const GbPool& pool, const GbParents& par, const ChildCtx& c,
                                               const GbSplit& sp) {
    const double* b = par.bnd + (size_t)c.p * sp.dmax * (sp.m + 1);
    return View<double>{pool.lo64 + (size_t)c.slot * pool.n, pool.hi64 + (size_t)c.slot * pool.n, b, b,
                        c.info.x, c.info.y, sp.mshift, sp.m + 1, c.r};
}
__device__ __forceinline__ View<float> view32(const GbPool& pool, const GbParents& par, const ChildCtx& c,
                                              const GbSplit& sp) {
    size_t o = (size_t)c.p * sp.dmax * (sp.m + 1);
    return View<float>{pool.lo32 + (size_t)c.slot * pool.n, pool.hi32 + (size_t)c.slot * pool.n,
                       par.bnd_rd + o, par.bnd_ru + o, c.info.x, c.info.y, sp.mshift, sp.m + 1, c.r};
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


}  // namespace gb
