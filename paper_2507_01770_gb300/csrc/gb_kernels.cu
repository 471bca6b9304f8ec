// Solver kernels: one generation of the batched best-first interval branch
// and bound (section 3.1 flowchart; partition of Eqs. 7-11 with the variable
// cycling of section 3.2), and the per-box evaluation used for parity.
//
// Generation, as launched by gb_api.cu:
//   stats      active count over the pool (LB < RU(GUB - tol_f), not final)
//   select     radix select of the K-th smallest LB key when active > K
//   partition  stable 3-way split of the pool: cut off (LB > GUB, section 3.1
//              "remove the suboptimal regions"), selected parents, kept
//   prep       per parent: the m+1 piece boundaries of each split coordinate
//   eval       per child: FP64 midpoint sample (GUB), F(X), first-order test;
//              or FP32 pass, compaction, FP64 pass on the FP32 survivors
//   compact    stable list of survivors (LB <= new GUB and not monotone)
//   materialize survivors written into free slots with their group caches
//   finish     parents' slots freed, counters rolled forward
// All orderings are deterministic (no atomics decide an order).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstdlib>

#include "gb_child.cuh"
#include "gb_eval.cuh"
#include "gb_launch.h"

using namespace gb;

namespace {

__device__ __forceinline__ double thr_of(double gub, double tol_f) { return __dsub_ru(gub, tol_f); }

// ---------------------------------------------------------------------------
// block-wide exclusive prefix of one flag per thread (item order = thread order)
template <int NT>
__device__ __forceinline__ int block_prefix(bool f, int* smem_warp, int* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned b = __ballot_sync(0xffffffffu, f);
    int in_warp = __popc(b & ((1u << lane) - 1u));
    if (lane == 0) smem_warp[wid] = __popc(b);
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int w = 0; w < NT / 32; w++) {
            int c = smem_warp[w];
            smem_warp[w] = acc;
            acc += c;
        }
        smem_warp[NT / 32] = acc;
    }
    __syncthreads();
    int r = smem_warp[wid] + in_warp;
    *total = smem_warp[NT / 32];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
// Root box: the whole domain [l, u] (section 3.1 "initialization").
template <bool PR>
__global__ void k_root_init(GbProg P, GbPool pool, GbEntries E, double tol_x, GbState* st) {
    const int n = P.n;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double l = P.l[j], u = P.u[j];
        // dense: slot 0's row; records: record b = j / B holds block b
        pool.recs ? (pool.rlo[j] = l) : (pool.lo64[j] = l);
        pool.recs ? (pool.rhi[j] = u) : (pool.hi64[j] = u);
        if (pool.fp32) {
            float l32 = __double2float_rd(l), u32 = __double2float_ru(u);
            pool.recs ? (pool.rlo32[j] = l32) : (pool.lo32[j] = l32);
            pool.recs ? (pool.rhi32[j] = u32) : (pool.hi32[j] = u32);
        }
    }
    if (pool.recs)
        for (int b = threadIdx.x; b < pool.nb; b += blockDim.x) {
            pool.rid[b] = (unsigned)b;
            bool wide = false;
            for (int j = b * pool.B; j < min(n, (b + 1) * pool.B); j++)
                if (!(__dsub_rn(P.u[j], P.l[j]) < tol_x)) wide = true;
            pool.rwide[b] = wide ? 1 : 0;
        }
    __syncthreads();
    if (pool.recs && threadIdx.x == 0) {
        int w = 0;
        for (int b = 0; b < pool.nb; b++) w += pool.rwide[b];
        pool.swide[0] = w;
    }
    View<double> X = box_view64(pool, 0);
    MidView MX{X};
    View<float> X32 = box_view32(pool, 0);
    iv64 R[GB_MAX_TREGS];
    iv32 R32[GB_MAX_TREGS];
    int ops = 0;
    for (int k = 0; k < P.n_sum; k++) {
        GbSum S = P.sums[k];
        for (int g = threadIdx.x; g < S.ngroups; g += blockDim.x) {
            const int gg = S.group0 + g;
            const size_t at = pool.recs ? (size_t)P.gown[gg].x * pool.GPB + P.gown[gg].y : (size_t)gg;
            iv64 a = group_sum<PR, double>(P, S, g, X, R, ops);
            iv64 b = group_sum<PR, double>(P, S, g, MX, R, ops);
            (pool.recs ? pool.rgsum : pool.gsum)[at] = make_double2(a.lo, a.hi);
            (pool.recs ? pool.rgmid : pool.gmid)[at] = make_double2(b.lo, b.hi);
            if (pool.fp32) {
                iv32 c = group_sum<PR, float>(P, S, g, X32, R32, ops);
                (pool.recs ? pool.rgsum32 : pool.gsum32)[at] = make_float2(c.lo, c.hi);
            }
            for (int j = 1; has_samp(pool) && j <= pool.S; j++) {
                const iv64 v = group_sum<PR, double>(P, S, g, SampleView{X, j, pool.S + 1}, R, ops);
                if (pool.recs) pool.rgsamp[(size_t)(j - 1) * pool.R * pool.GPB + at] = make_double2(v.lo, v.hi);
                else pool.gsamp[(size_t)(j - 1) * pool.NG + gg] = make_double2(v.lo, v.hi);
            }
        }
    }
    if (pool.gdp) {   // coordinate partials of the domain, every block
        iv64 RA[GB_MAX_TREGS];
        for (int b = threadIdx.x; b < P.nb; b += blockDim.x) block_D(P, b, X, R, RA, pool.gdp, n, 0, ops);
    }
    if (pool.rgdp) {   // the same per block record (the root's record of block b is b)
        iv64 RA[GB_MAX_TREGS];
        for (int b = threadIdx.x; b < P.nb; b += blockDim.x)
            block_D(P, b, X, R, RA, pool.rgdp + (size_t)b * P.n_sum * pool.B, pool.B, b * pool.B, ops);
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    // F and the midpoint sample from the group sums just cached (the same
    // group values and tree as a full evaluation)
    iv64 sums[GB_MAX_ISUM], O[GB_MAX_OREGS];
    const CacheRef<double2> cf = cache64(pool, P, 0, 0), cm = cache64(pool, P, 0, 1);
    sum_values<PR, double>(P, -1, X, &cf, R, sums, ops);
    iv64 F = outer_fwd<double>(P, X, sums, O, ops);
    double gub = __longlong_as_double(0x7ff0000000000000LL);
    long long nsamp = 1;
    if (P.samples > 0) {   // diagonal samples of the domain
        nsamp = P.samples;
        for (int j = 1; j <= P.samples; j++) {
            const SampleView SV{X, j, P.samples + 1};
            const CacheRef<double2> cs = samp64(pool, P, 0, j);
            sum_values<PR, double>(P, -1, SV, has_samp(pool) ? &cs : (const CacheRef<double2>*)nullptr, R, sums, ops);
            const iv64 Fs = outer_fwd<double>(P, SV, sums, O, ops);
            if (Fs.hi < gub) gub = Fs.hi;
        }
    } else {
        sum_values<PR, double>(P, -1, MX, &cm, R, sums, ops);
        const iv64 Fm = outer_fwd<double>(P, MX, sums, O, ops);
        if (Fm.hi == Fm.hi) gub = Fm.hi;
    }
    E.flo[0] = canon_lo(F.lo);
    E.slot[0] = 0;
    E.cyc[0] = 0;
    GbState s0 = {};
    s0.pool = 1;
    s0.nfree = 0;
    s0.bump = 1;
    s0.cap = st->cap;
    s0.gub_key = gb_order_key(gub);
    s0.gub_new_key = s0.gub_key;
    s0.sel_T = ~0ull;
    s0.min_key = ~0ull;
    s0.evals64 = 1;
    s0.mids = nsamp;
    s0.rec_bump = pool.recs ? pool.nb : 0;
    *st = s0;
}

// ---------------------------------------------------------------------------
// Every kernel of a generation reads its sizes (pool size, parents, children)
// and the incumbent GUB from the device state, so the launch sequence of a
// generation is fixed and can be replayed from a CUDA graph; a generation that
// must not run (no active box, limit reached, overflow, error) is skipped by
// every kernel through st->halt.

__device__ __forceinline__ double gub_of(const GbState* st) { return gb_key_value(st->gub_key); }

// Parents' slots back to the free list, or (on overflow) the parents back
// into the pool after the carried-over entries.
__device__ __forceinline__ void free_parents(const GbParents& par, const GbPool& pool, const GbEntries& En,
                                             const GbState* st, long long p0, long long step) {
    const long long npar = st->parents;
    for (long long p = p0; p < npar; p += step) {
        if (st->overflow) {
            long long e = st->kept_old + p;
            En.flo[e] = par.flo[p];
            En.slot[e] = par.slot[p];
            En.cyc[e] = par.cyc[p];
            continue;
        }
        long long kept = st->kept, nfree = st->nfree;
        long long base = kept < nfree ? nfree - kept : 0;
        pool.freel[base + p] = par.slot[p];
    }
}

// End of a generation, by the last block of k_stats: pool size, free list,
// record counters, GUB, trace row, generation number.
__device__ __forceinline__ void finish_counters(const GbGenConst& G, GbState* st) {
    const long long npar = st->parents;
    long long kept = st->kept, nfree = st->nfree;
    if (st->overflow) {
        st->pool = st->kept_old + npar;
        st->kept = 0;
    } else {
        long long from_free = kept < nfree ? kept : nfree;
        st->bump += kept - from_free;
        if (G.nrec) {
            const long long used = kept * G.nrec, rf = st->rec_nfree;
            const long long r_from_free = used < rf ? used : rf;
            st->rec_nfree = rf - r_from_free;
            st->rec_bump += used - r_from_free;
        }
        st->nfree = nfree - from_free + npar;
        st->pool = st->kept_old + kept;
    }
    st->gub_key = st->gub_new_key;
    if (G.trace && st->gen < G.trace_cap) {
        gb_gen_stat row;
        row.parents = npar;
        row.children = st->children;
        row.kept32 = G.fp32 ? st->kept32 : st->children;
        row.kept = st->overflow ? 0 : st->kept;
        row.pool = st->pool;
        row.gub = gb_key_value(st->gub_key);
        G.trace[st->gen] = row;
    }
    st->gen += 1;
    st->min_key = ~0ull;
    if (st->gc) st->rec_gc += 1;
    st->gc = 0;
}

// Pool statistics at the end of a generation (and after the root): the
// number of active entries and, for K = 1, the smallest active key and the
// last pool position holding it (the entry the selection takes: ties go to
// the most recently inserted).  Each block leaves its (key, position) pair;
// the last block to finish combines them and starts the next generation
// (open_generation).  With K = 1 the end of a generation does not need this
// pass over the pool: the partition and k_materialize leave the pairs of the
// entries they write, and k_materialize's last block does the rest.
__device__ __forceinline__ void better_key(unsigned long long& k, long long& q, unsigned long long k2, long long q2) {
    if (k2 < k || (k2 == k && q2 > q)) k = k2, q = q2;
}

// The best (key, position) pair of a block; every thread calls it, thread 0
// gets the result (sk, sq: one entry per warp in shared memory).
__device__ __forceinline__ void block_best(unsigned long long& k, long long& q, unsigned long long* sk, long long* sq) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o; o >>= 1) {
        const unsigned long long k2 = __shfl_down_sync(0xffffffffu, k, o);
        const long long q2 = __shfl_down_sync(0xffffffffu, q, o);
        better_key(k, q, k2, q2);
    }
    __syncthreads();
    if (lane == 0) sk[w] = k, sq[w] = q;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int i = 1; i < (int)(blockDim.x >> 5); i++) better_key(k, q, sk[i], sq[i]);
}

// The best pair over n per-block pairs (every thread of one block calls it;
// thread 0 gets the result).
__device__ __forceinline__ void combine_pairs(const unsigned long long* bkey, const long long* bpos, int n,
                                              unsigned long long& k, long long& q, unsigned long long* sk,
                                              long long* sq) {
    k = ~0ull;
    q = -1;
    for (int b = threadIdx.x; b < n; b += blockDim.x) better_key(k, q, __ldcg(bkey + b), __ldcg(bpos + b));
    block_best(k, q, sk, sq);
}

// By one thread, once the new pool's active count and (for K = 1) its
// smallest active key mk and that key's last position mq are known: stop
// the solve if nothing is active or a limit was reached, else choose the
// next selection (K = 1: the entry at mq; all active entries if at most K;
// else a radix select of the K-th smallest key) and open the next pool
// partition (ticket 0, a new epoch).
__device__ __forceinline__ void open_generation(const GbGenConst& G, GbState* st, long long active,
                                                unsigned long long mk, long long mq) {
    st->nfree_base = st->nfree;
    st->stats_done = 0;
    st->part_ticket = 0;
    st->part_epoch += 1;
    st->active = active;
    if (active == 0 || st->gen >= G.max_gen || st->overflow || st->error) {
        st->halt = 1;
        return;
    }
    if (G.K == 1) {
        // the smallest active key, the most recently inserted entry holding it
        st->sel_mode = 1;
        st->sel_T = mk;
        st->sel_pos = mq;
        st->sel_below = 0;
        st->sel_need = 1;
    } else if (active <= G.K) {
        st->sel_mode = 0;
        st->sel_T = ~0ull;
        st->sel_below = active;
        st->sel_need = 0;
    } else {
        st->sel_mode = 2;
        st->radix_prefix = 0;
        st->radix_rank = G.K;
        st->sel_below = 0;
    }
}

__global__ void __launch_bounds__(256) k_stats(GbEntries E, GbGenConst G, GbState* st, unsigned long long* bkey,
                                               long long* bpos, GbParents par, GbPool pool, int finish) {
    gb_grid_trigger();
    gb_grid_wait();
    if (st->halt) return;
    __shared__ unsigned long long s_c[8], s_k[8];
    __shared__ long long s_q[8];
    __shared__ bool s_last;
    // at the end of a generation (finish): the parents' slots go back to the
    // free list (on overflow the parents go back into the pool), and the new
    // pool and incumbent are read from the generation's counters; the last
    // block rolls the counters forward
    if (finish) free_parents(par, pool, E, st, blockIdx.x * (long long)blockDim.x + threadIdx.x,
                             (long long)gridDim.x * blockDim.x);
    const long long count = !finish ? st->pool
                                    : st->kept_old + (st->overflow ? st->parents : st->kept);
    const double thr = thr_of(gb_key_value(finish ? st->gub_new_key : st->gub_key), G.tol_f);
    long long c = 0, kq = -1;
    unsigned long long kmin = ~0ull;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < count;
         q += (long long)gridDim.x * blockDim.x) {
        const double f = E.flo[q];
        if (f < thr && !((unsigned)E.cyc[q] & GB_FINAL_BIT)) {
            c++;
            better_key(kmin, kq, gb_order_key(f), q);
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o; o >>= 1) {
        c += __shfl_down_sync(0xffffffffu, c, o);
        const unsigned long long k2 = __shfl_down_sync(0xffffffffu, kmin, o);
        const long long q2 = __shfl_down_sync(0xffffffffu, kq, o);
        better_key(kmin, kq, k2, q2);
    }
    if (lane == 0) s_c[w] = (unsigned long long)c, s_k[w] = kmin, s_q[w] = kq;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long tc = 0, tk = ~0ull;
        long long tq = -1;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) tc += s_c[i], better_key(tk, tq, s_k[i], s_q[i]);
        if (tc) atomicAdd((unsigned long long*)&st->active_acc, tc);
        bkey[blockIdx.x] = tk;
        bpos[blockIdx.x] = tq;
    }
    if (!arrive_last(&st->stats_done, gridDim.x, &s_last)) return;
    // last block: combine every block's pair, then start the next generation
    kmin = ~0ull;
    kq = -1;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) better_key(kmin, kq, __ldcg(bkey + b), __ldcg(bpos + b));
    for (int o = 16; o; o >>= 1) {
        const unsigned long long k2 = __shfl_down_sync(0xffffffffu, kmin, o);
        const long long q2 = __shfl_down_sync(0xffffffffu, kq, o);
        better_key(kmin, kq, k2, q2);
    }
    if (lane == 0) s_k[w] = kmin, s_q[w] = kq;
    __syncthreads();
    if (threadIdx.x != 0) return;
    unsigned long long mk = ~0ull;
    long long mq = -1;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) better_key(mk, mq, s_k[i], s_q[i]);
    if (finish) finish_counters(G, st);
    const long long active = (long long)atomicExch((unsigned long long*)&st->active_acc, 0ull);
    open_generation(G, st, active, mk, mq);
}

// Radix select (16-bit digits, 4 passes) of the K-th smallest active key.
__global__ void k_radix_hist(GbEntries E, GbGenConst G, int pass, const GbState* st, unsigned* hist) {
    if (st->halt || st->sel_mode != 2) return;
    const long long count = st->pool;
    const double thr = thr_of(gub_of(st), G.tol_f);
    const unsigned long long prefix = st->radix_prefix;
    const int shift = 48 - 16 * pass;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < count;
         q += (long long)gridDim.x * blockDim.x) {
        double f = E.flo[q];
        if (!(f < thr) || ((unsigned)E.cyc[q] & GB_FINAL_BIT)) continue;
        unsigned long long key = gb_order_key(f);
        if (pass > 0 && (key >> (shift + 16)) != prefix) continue;
        atomicAdd(&hist[(key >> shift) & 0xffffu], 1u);
    }
}

// One block of 1024 threads (32 warps, each owning 2048 consecutive bins):
// coalesced warp totals, a scan over the 32 totals, then the owning warp
// walks its chunk 32 bins at a time.  Clears the histogram for the next pass.
__global__ void __launch_bounds__(1024) k_radix_pick(int pass, GbState* st, unsigned* hist) {
    if (st->halt || st->sel_mode != 2) return;
    __shared__ long long wtot[32];
    __shared__ long long wpre[33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned* h = hist + w * 2048;
    long long s = 0;
    for (int k = 0; k < 64; k++) s += h[k * 32 + lane];
    for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) wtot[w] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long acc = 0;
        for (int i = 0; i < 32; i++) {
            wpre[i] = acc;
            acc += wtot[i];
        }
        wpre[32] = acc;
    }
    __syncthreads();
    const long long rank = st->radix_rank;
    if (wpre[w] < rank && rank <= wpre[w] + wtot[w]) {
        long long acc = wpre[w];
        for (int k = 0; k < 64; k++) {
            long long c = h[k * 32 + lane];
            long long inc = c;
            for (int o = 1; o < 32; o <<= 1) {
                long long v = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += v;
            }
            long long before = acc + inc - c;   // bins before this lane's bin
            bool hit = before < rank && rank <= before + c;
            unsigned b = __ballot_sync(0xffffffffu, hit);
            if (hit) {
                st->radix_prefix = (st->radix_prefix << 16) | (unsigned long long)(w * 2048 + k * 32 + lane);
                st->radix_rank = rank - before;
                st->sel_below += before;
                if (pass == 3) st->sel_ties = c;   // entries whose whole key equals the threshold
            }
            if (b) break;
            acc += __shfl_sync(0xffffffffu, inc, 31);
        }
    }
    __syncthreads();
    for (int k = 0; k < 64; k++) hist[w * 2048 + k * 32 + lane] = 0;
    if (threadIdx.x == 0 && pass == 3) {
        st->sel_T = st->radix_prefix;
        st->sel_need = st->radix_rank;
        if (wpre[32] < rank) st->error |= 1;
    }
}

// ---------------------------------------------------------------------------
// Pool partition: class of an entry (cut off, selected below the threshold,
// tie at the threshold).
struct PartFlags { bool drop, below, tie; };

constexpr int PT = 256;  // threads per partition / compaction block; tile = 4 rounds

__device__ __forceinline__ long long ntiles_of(long long items) { return (items + GB_TILE - 1) / GB_TILE; }

// Survivor count S of the generation: overflow if the slots cannot take
// them; with block records, a collection first if their new records do not fit.

// Exclusive scan of an array of tile counts (one block of 1024 threads,
// each owning a contiguous run of tiles).
// what: 1 = FP32 list and 2 = survivors (items = children of the
// generation), 3 = output (items = count), 4 = free block records (items =
// records ever used).
__global__ void __launch_bounds__(1024) k_scan_tiles(int narr, const int* tile_cnt, int* tile_off, int max_tiles,
                                                     int what, long long out_count, GbGenConst G, GbState* st) {
    gb_grid_trigger();
    gb_grid_wait();
    if (what != 3 && st->halt) return;
    if (what == 4 && !st->gc) return;
    __shared__ long long part[1024];
    __shared__ long long tot[3];
    const long long items = what == 3 ? out_count : what == 4 ? st->rec_bump : st->nch;
    const int ntiles = (int)ntiles_of(items);
    const int t = threadIdx.x;
    const int per = (ntiles + 1023) / 1024;
    for (int a = 0; a < narr; a++) {
        const int* c = tile_cnt + a * max_tiles;
        int* o = tile_off + a * max_tiles;
        int i0 = t * per, i1 = min(ntiles, i0 + per);
        long long s = 0;
        for (int i = i0; i < i1; i++) s += c[i];
        part[t] = s;
        __syncthreads();
        for (int d = 1; d < 1024; d <<= 1) {
            long long v = t >= d ? part[t - d] : 0;
            __syncthreads();
            part[t] += v;
            __syncthreads();
        }
        long long acc = part[t] - s;
        for (int i = i0; i < i1; i++) {
            o[i] = (int)acc;
            acc += c[i];
        }
        if (t == 1023) tot[a] = part[1023];
        __syncthreads();
    }
    if (t != 0) return;
    if (what == 1) {
        st->n32 = tot[0];
        st->kept32 = tot[0];
    } else if (what == 2) {
        set_survivors(G, st, tot[0]);
    } else if (what == 4) {
        st->rec_nfree = tot[0];
    } else {
        st->kept = tot[0];
    }
}

// Pool partition in one launch.  Tiles of GB_TILE entries are handed out in
// order (a ticket); each tile classifies its entries (cut off, selected --
// below the threshold, or the K = 1 entry --, tie), publishes its three
// counts, finds the counts of every tile before it by looking back at their
// published values (decoupled look-back: a predecessor's inclusive prefix
// ends the walk, its aggregate is added and the walk goes on), publishes its
// own inclusive prefix and scatters its entries stably: cut-off slots to the
// free list, parents to the parent buffers (the last `need` ties in pool
// order), the rest to the new pool.  A tile only waits for tiles whose
// tickets were taken before its own, by blocks already running, so every
// wait ends; each is bounded all the same (on running out it sets an error
// bit and publishes, so no block waits on it).  The tile that finishes last
// in order writes the totals of the partition.  With par_by_tab (K = 1 and
// term tables) the single parent is written by k_ptab, which reads it from
// the pool position k_stats found and may run at the same time.
constexpr unsigned long long GB_FLAG_AGG = 1, GB_FLAG_INC = 2;
constexpr long long GB_SPIN_LIMIT = 1LL << 26;

__device__ __forceinline__ PartFlags part_flags1(const GbEntries& E, long long q, long long count, double gub,
                                                 double thr, unsigned long long T, int mode, long long spos) {
    PartFlags f{false, false, false};
    if (q >= count) return f;
    const double v = E.flo[q];
    if (v > gub) { f.drop = true; return f; }
    const bool act = v < thr && !((unsigned)E.cyc[q] & GB_FINAL_BIT);
    if (!act) return f;
    if (mode == 1) { f.below = q == spos; return f; }
    if (T == ~0ull) { f.below = true; return f; }
    const unsigned long long key = gb_order_key(v);
    f.below = key < T;
    f.tie = key == T;
    return f;
}

// Exclusive block scan of one 64-bit value per thread (PT threads; packed
// counters add field by field as long as no field overflows); the block's
// total is left in sh[PT / 32].
__device__ __forceinline__ unsigned long long block_scan_packed(unsigned long long v, unsigned long long* sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) sh[w] = inc;
    __syncthreads();
    if (w == 0) {
        unsigned long long x = lane < PT / 32 ? sh[lane] : 0, xi = x;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += y;
        }
        if (lane < PT / 32) sh[lane] = xi - x;   // exclusive warp offsets
        if (lane == PT / 32 - 1) sh[PT / 32] = xi;
    }
    __syncthreads();
    return sh[w] + inc - v;
}

__global__ void __launch_bounds__(PT) k_part_1p(GbEntries E, GbGenConst G, GbState* st, int* agg, int* inc,
                                                int max_tiles, unsigned long long* flag, GbEntries En,
                                                GbParents par, unsigned* freel, int par_by_tab,
                                                unsigned long long* pkey, long long* ppos) {
    gb_grid_trigger();
    gb_grid_wait();
    if (st->halt) return;
    __shared__ unsigned long long s_scan[PT / 32 + 1], s_bk[PT / 32];
    __shared__ long long s_bq[PT / 32];
    __shared__ long long s_tile;
    __shared__ long long s_ex[3];
    const long long count = st->pool;
    const double gub = gub_of(st);
    const double thr = thr_of(gub, G.tol_f);
    const int mode = st->sel_mode;
    const unsigned long long T = st->sel_T;
    const long long spos = st->sel_pos;
    // ties (key == T) exist only for the radix threshold; the last `need` of them are taken
    const long long need = (mode == 2 && T != ~0ull) ? st->sel_need : 0;
    const long long Ti = (mode == 2 && T != ~0ull) ? st->sel_ties : 0;
    // (st->nfree itself is rewritten by the last tile while late blocks start)
    const long long nfree = st->nfree_base;
    const unsigned long long epoch = st->part_epoch;
    const long long nt = ntiles_of(count);
    auto totals = [&](long long D, long long Bl, long long Tt) {
        const long long npar = Bl + need;
        st->drops = D;
        st->parents = npar;
        st->nch = npar << G.flog2;
        st->kept_old = count - D - npar;
        st->nfree = nfree + D;
        st->sel_below = Bl;
        st->sel_ties = Tt;
        // a record collection when the generation's children might not fit
        st->gc = (G.nrec && (npar << G.flog2) * G.nrec > st->rec_nfree + (G.R - st->rec_bump)) ? 1 : 0;
    };
    if (nt == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) totals(0, 0, 0);
        if (pkey && blockIdx.x == 0 && threadIdx.x == 0) pkey[0] = ~0ull, ppos[0] = -1;
        return;
    }
    // pkey: the smallest key of the kept entries that can be selected (not
    // final) and its last new position: one pair per block, combined into
    // pkey[0] by the last block to finish
    unsigned long long bk = ~0ull;
    long long bq = -1;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_tile = (long long)atomicAdd(&st->part_ticket, 1ull);
        __syncthreads();
        const long long tile = s_tile;
        if (tile >= nt) break;
        const long long base = tile * GB_TILE;
        // thread t classifies entries base + 4t .. base + 4t + 3; the three
        // counts travel packed (21 bits each) through one block scan
        constexpr int PER = GB_TILE / PT;
        const long long q0 = base + (long long)PER * threadIdx.x;
        PartFlags f[PER];
#pragma unroll
        for (int u = 0; u < PER; u++) f[u] = part_flags1(E, q0 + u, count, gub, thr, T, mode, spos);
        unsigned long long mine = 0;
#pragma unroll
        for (int u = 0; u < PER; u++)
            mine += (unsigned long long)f[u].drop | ((unsigned long long)f[u].below << 21) |
                    ((unsigned long long)f[u].tie << 42);
        const unsigned long long before = block_scan_packed(mine, s_scan);   // exclusive
        const unsigned long long total = s_scan[PT / 32];
        int rd[PER], rb[PER], rt[PER];
        {
            unsigned long long run = before;
#pragma unroll
            for (int u = 0; u < PER; u++) {
                rd[u] = (int)(run & 0x1fffff);
                rb[u] = (int)((run >> 21) & 0x1fffff);
                rt[u] = (int)(run >> 42);
                run += (unsigned long long)f[u].drop | ((unsigned long long)f[u].below << 21) |
                       ((unsigned long long)f[u].tie << 42);
            }
        }
        const int cd = (int)(total & 0x1fffff), cb = (int)((total >> 21) & 0x1fffff), ct = (int)(total >> 42);
        // publication and look-back by warp 0: its lanes inspect 32
        // predecessors at a time (the nearest inclusive prefix ends the walk,
        // the aggregates after it are summed)
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            volatile unsigned long long* vf = flag;
            volatile int* va = agg;
            volatile int* vi = inc;
            long long ed = 0, eb = 0, et = 0;
            if (tile > 0) {
                if (lane == 0) {
                    agg[tile] = cd;
                    agg[max_tiles + tile] = cb;
                    agg[2 * max_tiles + tile] = ct;
                    __threadfence();
                    vf[tile] = (epoch << 2) | GB_FLAG_AGG;
                }
                bool bad = false, done = false;
                long long top = tile - 1;   // the window is [top - 31, top]
                while (!done) {
                    const long long j = top - lane;
                    unsigned long long fl = epoch << 2 | GB_FLAG_INC;   // lanes before tile 0: an empty prefix
                    long long spins = 0;
                    if (j >= 0)
                        while (((fl = vf[j]) >> 2) != epoch)
                            if (++spins > GB_SPIN_LIMIT) { bad = true; break; }
                    if (__any_sync(0xffffffffu, bad)) { bad = true; break; }
                    __threadfence();
                    const unsigned incm = __ballot_sync(0xffffffffu, (fl & 3) == GB_FLAG_INC);
                    const int stop = incm ? __ffs(incm) - 1 : 31;   // the nearest inclusive prefix (or the window end)
                    long long xd = 0, xb = 0, xt = 0;
                    if (j >= 0 && lane <= stop) {
                        const bool isinc = (fl & 3) == GB_FLAG_INC;
                        const volatile int* vs = isinc ? vi : va;
                        xd = vs[j];
                        xb = vs[max_tiles + j];
                        xt = vs[2 * max_tiles + j];
                    }
                    for (int o = 16; o; o >>= 1) {
                        xd += __shfl_down_sync(0xffffffffu, xd, o);
                        xb += __shfl_down_sync(0xffffffffu, xb, o);
                        xt += __shfl_down_sync(0xffffffffu, xt, o);
                    }
                    ed += __shfl_sync(0xffffffffu, xd, 0);
                    eb += __shfl_sync(0xffffffffu, xb, 0);
                    et += __shfl_sync(0xffffffffu, xt, 0);
                    done = incm != 0 || top - 31 < 0;
                    top -= 32;
                }
                if (bad && lane == 0) atomicOr(&st->error, 4);
            }
            if (lane == 0) {
                inc[tile] = (int)(ed + cd);
                inc[max_tiles + tile] = (int)(eb + cb);
                inc[2 * max_tiles + tile] = (int)(et + ct);
                __threadfence();
                vf[tile] = (epoch << 2) | GB_FLAG_INC;
                s_ex[0] = ed;
                s_ex[1] = eb;
                s_ex[2] = et;
                if (tile == nt - 1) totals(ed + cd, eb + cb, et + ct);
            }
        }
        __syncthreads();
        const long long od = s_ex[0], ob = s_ex[1], ot = s_ex[2];
#pragma unroll
        for (int r = 0; r < PER; r++) {
            const long long q = q0 + r;
            if (q >= count) continue;
            const long long gd = od + rd[r], gb = ob + rb[r], gt = ot + rt[r];
            const long long sel_before = gb + max(0LL, gt - (Ti - need));
            const bool sel = f[r].below || (f[r].tie && gt >= Ti - need);
            if (f[r].drop) {
                freel[nfree + gd] = E.slot[q];
            } else if (sel) {
                if (par_by_tab) continue;   // the table kernel writes the single parent
                par.slot[sel_before] = E.slot[q];
                par.cyc[sel_before] = E.cyc[q];
                par.flo[sel_before] = E.flo[q];
            } else {
                const long long kr = q - gd - sel_before;
                const double v = E.flo[q];
                const int cy = E.cyc[q];
                En.flo[kr] = v;
                En.slot[kr] = E.slot[q];
                En.cyc[kr] = cy;
                if (!((unsigned)cy & GB_FINAL_BIT)) better_key(bk, bq, gb_order_key(v), kr);
            }
        }
    }
    if (!pkey) return;
    __shared__ bool s_last;
    block_best(bk, bq, s_bk, s_bq);
    if (threadIdx.x == 0) {
        pkey[blockIdx.x] = bk;
        ppos[blockIdx.x] = bq;
    }
    if (!arrive_last(&st->part_done, gridDim.x, &s_last)) return;
    combine_pairs(pkey, ppos, (int)gridDim.x, bk, bq, s_bk, s_bq);
    if (threadIdx.x == 0) {
        pkey[0] = bk;
        ppos[0] = bq;
        st->part_done = 0;
    }
}

// ---------------------------------------------------------------------------
// Per parent: split coordinates and piece boundaries (Eqs. 10-11 with the
// rounding reading: boundary t = RN(lo + RN(RN(RN(hi - lo) / m) * t)),
// boundary 0 = lo, boundary m = hi).
// One thread per (parent, split coordinate): the split position of the
// parent and the piece boundaries of one coordinate (the divisions of the
// coordinates run in parallel).
__global__ void k_prep(GbProg P, GbPool pool, GbParents par, GbSplit sp, GbState* st) {
    if (st->halt) return;
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx == 0) {
        st->gub_new_key = st->gub_key;
        st->kept = 0;
        st->kept32 = 0;
        st->n32 = 0;
        st->children = 0;
        st->overflow = 0;
    }
    const long long npar = st->parents;
    const long long p = idx / sp.dmax;
    const int k = (int)(idx - p * sp.dmax);
    if (p >= npar) return;
    const int n = P.n, B = P.B;
    int c = par.cyc[p] & 0x7fffffff;
    int b = c / B;
    int e = min((b + 1) * B, n);
    int dd = min(sp.d, e - c);
    int nxt = (c + dd == n) ? 0 : c + dd;
    if (k == 0) par.info[p] = make_int4(c, dd, b, nxt);
    unsigned slot = par.slot[p];
    const int ms = sp.m + 1;
    const View<double> PX = box_view64(pool, slot);
    if (k < dd) {
        int j = c + k;
        const iv64 pj = PX.get(j);
        double lo = pj.lo, hi = pj.hi;
        double w = __dsub_rn(hi, lo);
        double q = __ddiv_rn(w, (double)sp.m);
        for (int t = 0; t <= sp.m; t++) {
            double v = (t == 0) ? lo : (t == sp.m ? hi : __dadd_rn(lo, __dmul_rn(q, (double)t)));
            size_t o = ((size_t)p * sp.dmax + k) * ms + t;
            par.bnd[o] = v;
            par.bnd_rd[o] = __double2float_rd(v);
            par.bnd_ru[o] = __double2float_ru(v);
        }
    }
}

// FP64 child evaluation: midpoint sample, F(X), first-order test.
// First-order test: the active block, or every block (mono_all).
// gc: the parent's cached group values (groups dirty for blk recomputed).
template <bool PR, typename T, typename V, typename C>
__device__ __forceinline__ bool mono_any(const GbProg& P, int blk, const V& X, const View<double>& X64,
                                         const typename Prec<T>::I* O, typename Prec<T>::I* OA,
                                         typename Prec<T>::I* R, typename Prec<T>::I* RA,
                                         const CacheRef<C>* gc, int& ops) {
    if (!P.mono_all) return block_mono<PR, T>(P, blk, X, X64, O, OA, R, RA, (double*)nullptr, gc, blk, ops);
    for (int b = 0; b < P.nb; b++)
        if (block_mono<PR, T>(P, b, X, X64, O, OA, R, RA, (double*)nullptr, gc, blk, ops)) return true;
    return false;
}

// First-order test on every coordinate with the parent's cached D: the
// blocks a split of blk changes are tested in full, every other block from
// the cache with the child's own outer adjoints (the same operations in the
// same order as the full test, so the same decision).
template <typename V>
__device__ __noinline__ bool mono_cached(const GbProg& P, const GbPool& pool, unsigned slot, int blk, const V& X,
                                         const iv64* O, iv64* OA, iv64* R, iv64* RA, int& ops) {
    const int2 ab = d_affected(P, blk);
    for (int b = ab.x; b <= ab.y; b++)   // also leaves the outer adjoints in OA
        if (block_mono<false, double>(P, b, X, X, O, OA, R, RA, (double*)nullptr, (const CacheRef<double2>*)nullptr, -1,
                               ops))
            return true;
    for (int b = 0; b < P.nb; b++) {
        if (b >= ab.x && b <= ab.y) continue;
        // dense: the box's row; records: the parent's record of block b
        const bool hit = pool.recs
            ? cached_mono(P, b, X, OA,
                          pool.rgdp + (size_t)pool.rid[(size_t)slot * pool.nb + b] * P.n_sum * pool.B, pool.B,
                          b * pool.B, ops)
            : cached_mono(P, b, X, OA, pool.gdp + (size_t)slot * P.n_sum * P.n, P.n, 0, ops);
        if (hit) return true;
    }
    return false;
}

template <bool PR>
__device__ __forceinline__ bool eval64_child(const GbProg& P, const GbPool& pool, const GbParents& par,
                                             const GbChildren& ch, long long ci, const GbSplit& sp,
                                             double gub_prev, unsigned long long* gkey, bool* has_key,
                                             int& ops) {
    ChildCtx c = child_ctx(par, ci, sp);
    if (!c.valid) {
        ch.flag[ci] = 0;
        ch.flo[ci] = __longlong_as_double(0x7ff0000000000000LL);
        return false;
    }
    View<double> X = view64(pool, par, c, sp);
    MidView MX{X};
    iv64 R[GB_MAX_TREGS], RA[GB_MAX_TREGS], O[GB_MAX_OREGS], OA[GB_MAX_OREGS], sums[GB_MAX_ISUM];
    const int blk = c.info.z;
    const CacheRef<double2> cm = cache64(pool, P, c.slot, 1), cf = cache64(pool, P, c.slot, 0);
    if (P.samples > 0) {   // diagonal samples, each evaluated in full
        for (int j = 1; j <= P.samples; j++) {
            const SampleView SV{X, j, P.samples + 1};
            // the child's sample j agrees with its parent's on every coordinate
            // it did not split: the groups off the split block come from the cache
            const CacheRef<double2> cs = samp64(pool, P, c.slot, j);
            sum_values<PR, double>(P, blk, SV, has_samp(pool) ? &cs : (const CacheRef<double2>*)nullptr, R, sums, ops);
            const iv64 Fs = outer_fwd<double>(P, SV, sums, O, ops);
            if (Fs.hi == Fs.hi) {
                const unsigned long long k = gb_order_key(Fs.hi);
                if (!*has_key || k < *gkey) *gkey = k;
                *has_key = true;
            }
        }
    } else {
        sum_values<PR, double>(P, blk, MX, &cm, R, sums, ops);
        iv64 Fm = outer_fwd<double>(P, MX, sums, O, ops);
        if (Fm.hi == Fm.hi) {
            *gkey = gb_order_key(Fm.hi);
            *has_key = true;
        }
    }
    sum_values<PR, double>(P, blk, X, &cf, R, sums, ops);
    iv64 F = outer_fwd<double>(P, X, sums, O, ops);
    bool keep = !(F.lo > gub_prev);
    if (keep)
        keep = !(pool.gdp || pool.rgdp ? mono_cached(P, pool, c.slot, blk, X, O, OA, R, RA, ops)
                          : mono_any<PR, double>(P, blk, X, X, O, OA, R, RA, &cf, ops));
    ch.flo[ci] = canon_lo(F.lo);
    ch.flag[ci] = keep ? 1 : 0;
    return true;
}

template <bool PR>
__global__ void __launch_bounds__(128) k_eval64(GbProg P, GbPool pool, GbParents par, GbChildren ch, GbSplit sp,
                                                int from_list, GbState* st) {
    if (st->halt) return;
    const long long lim = from_list ? st->n32 : st->nch;
    const double gub_prev = gub_of(st);
    const long long stride = (long long)gridDim.x * blockDim.x;
    // warp-uniform loop: every lane of a warp runs the same iterations
    for (long long base = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); base < lim; base += stride) {
        long long idx = base + (threadIdx.x & 31);
        unsigned long long key = ~0ull;
        bool has = false;
        bool valid = false;
        int ops = 0;
        if (idx < lim) {
            long long ci = from_list ? (long long)ch.list32[idx] : idx;
            valid = eval64_child<PR>(P, pool, par, ch, ci, sp, gub_prev, &key, &has, ops);
        }
        warp_min_gub(key, has, st);
        warp_add_ops(ops, &st->ops64);
        unsigned nv = __popc(__ballot_sync(0xffffffffu, valid));
        if ((threadIdx.x & 31) == 0 && nv) {
            atomicAdd((unsigned long long*)&st->evals64, (unsigned long long)nv);
            atomicAdd((unsigned long long*)&st->mids, (unsigned long long)nv * (P.samples > 0 ? P.samples : 1));
            if (!from_list) atomicAdd((unsigned long long*)&st->children, (unsigned long long)nv);
        }
    }
}

// FP32 prefilter: F(X) and the first-order test in FP32 directed rounding,
// cut-off against the GUB of the previous generation.
template <bool PR>
__global__ void __launch_bounds__(128) k_eval32(GbProg P, GbPool pool, GbParents par, GbChildren ch, GbSplit sp,
                                                GbState* st) {
    if (st->halt) return;
    const long long lim = st->nch;
    const double gub_prev = gub_of(st);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); base < lim; base += stride) {
        long long ci = base + (threadIdx.x & 31);
        bool valid = false;
        int ops = 0;
        if (ci < lim) {
            ChildCtx c = child_ctx(par, ci, sp);
            ch.flag[ci] = 0;
            ch.flo[ci] = __longlong_as_double(0x7ff0000000000000LL);
            if (c.valid) {
                valid = true;
                View<float> X = view32(pool, par, c, sp);
                View<double> X64 = view64(pool, par, c, sp);
                iv32 R[GB_MAX_TREGS], RA[GB_MAX_TREGS], O[GB_MAX_OREGS], OA[GB_MAX_OREGS], sums[GB_MAX_ISUM];
                const int blk = c.info.z;
                const CacheRef<float2> c32 = cache32(pool, P, c.slot);
                sum_values<PR, float>(P, blk, X, &c32, R, sums, ops);
                iv32 F = outer_fwd<float>(P, X, sums, O, ops);
                bool keep = !((double)F.lo > gub_prev);
                if (keep) keep = !mono_any<PR, float>(P, blk, X, X64, O, OA, R, RA, &c32, ops);
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
// Stable compaction of child indices by a predicate (3 phases).
__device__ __forceinline__ bool child_pred(const GbChildren& ch, long long i, long long n, int mode,
                                           double gub_new) {
    if (i >= n) return false;
    if (mode == 0) return ch.flag32[i] != 0;
    return ch.flag[i] != 0 && !(ch.flo[i] > gub_new);
}

__global__ void k_cc_count(GbChildren ch, int mode, const GbState* st, int* tile_cnt) {
    gb_grid_trigger();
    gb_grid_wait();
    if (st->halt) return;
    __shared__ int sw[PT / 32 + 1];
    const long long n = st->nch;
    const double gub_new = gb_key_value(st->gub_new_key);
    const long long nt = ntiles_of(n);
    for (long long tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        const long long base = tile * GB_TILE;
        int acc = 0, tot;
        for (int r = 0; r < GB_TILE / PT; r++) {
            block_prefix<PT>(child_pred(ch, base + r * PT + threadIdx.x, n, mode, gub_new), sw, &tot);
            acc += tot;
        }
        if (threadIdx.x == 0) tile_cnt[tile] = acc;
    }
}

__global__ void k_cc_scatter(GbChildren ch, int mode, const GbState* st, const int* tile_off, unsigned* out) {
    gb_grid_trigger();
    gb_grid_wait();
    if (st->halt) return;
    __shared__ int sw[PT / 32 + 1];
    const long long n = st->nch;
    const double gub_new = gb_key_value(st->gub_new_key);
    const long long nt = ntiles_of(n);
    for (long long tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        const long long base = tile * GB_TILE;
        long long o = tile_off[tile];
        for (int r = 0; r < GB_TILE / PT; r++) {
            long long i = base + r * PT + threadIdx.x;
            bool f = child_pred(ch, i, n, mode, gub_new);
            int tot;
            int rk = block_prefix<PT>(f, sw, &tot);
            if (f) out[o + rk] = (unsigned)i;
            o += tot;
        }
    }
}

// Table path of the materialisation: the dirty group values of a survivor
// (F, midpoint, FP32), one warp walking the term-tree segments of its split
// position (warp_group), staged in shared memory at [k * GB_TAB_MAX_DIRTY +
// g - dr.x].
constexpr int GB_SHG = GB_MAX_ISUM * GB_TAB_MAX_DIRTY;
__device__ __forceinline__ void tab_dirty_groups(const GbProg& P, const GbPool& pool, const GbTabs& Tb,
                                                 const ChildCtx& c, long long ci, int lane, double2* shF,
                                                 double2* shM, float2* sh32) {
    if (Tb.cg64) {   // computed by k_child_sums: copy the slots
        for (int q = lane; q < GB_SHG; q += 32) {
            const size_t at = (size_t)ci * GB_CG + q;
            shF[q] = Tb.cg64[at];
            shM[q] = Tb.cgm64[at];
            if (pool.fp32) sh32[q] = Tb.cg32[at];
        }
        __syncwarp();
        return;
    }
    const GbSplitPos SP = P.sps[P.sp_of_cyc[c.info.x]];
    const int blk = c.info.z;
    const size_t rowbase = (size_t)c.p * Tb.max_rows, sbase = (size_t)c.p * Tb.max_srows;
    int dtA = SP.seg0, dtB = SP.seg0;
    for (int k = 0; k < P.n_sum; k++) {
        const int2 dr = P.dirty[blk * P.n_sum + k];
        for (int g = dr.x; g < dr.y; g++) {
            iv64 v2[2];
            int cnt;
            warp_group<iv64, 2>(P, SP, k, g, c.r, dtA, lane,
                                [&](const GbSeg& G, int at, iv64* v) {
                                    const double2 a = G.level ? Tb.ts64[sbase + at] : Tb.tv64[rowbase + at];
                                    const double2 b = G.level ? Tb.tsm64[sbase + at] : Tb.tm64[rowbase + at];
                                    v[0] = iv64{a.x, a.y};
                                    v[1] = iv64{b.x, b.y};
                                }, v2, cnt);
            const int at = k * GB_TAB_MAX_DIRTY + (g - dr.x);
            if (lane == 0) {
                shF[at] = make_double2(v2[0].lo, v2[0].hi);
                shM[at] = make_double2(v2[1].lo, v2[1].hi);
            }
            if (pool.fp32) {
                iv32 f;
                warp_group<iv32, 1>(P, SP, k, g, c.r, dtB, lane,
                                    [&](const GbSeg& G, int at, iv32* v) {
                                        const float2 a = G.level ? Tb.ts32[sbase + at] : Tb.tv32[rowbase + at];
                                        v[0] = iv32{a.x, a.y};
                                    }, &f, cnt);
                if (lane == 0) sh32[at] = make_float2(f.lo, f.hi);
            }
        }
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// Survivors into free slots: coordinates, FP32 shadow, group caches (dirty
// groups recomputed, the rest copied from the parent), pool entry.
template <bool PR, bool TAB>
__device__ __forceinline__ void materialize_one(const GbProg& P, const GbPool& pool, const GbParents& par,
                                                const GbChildren& ch, const GbSplit& sp, const GbEntries& En,
                                                double tol_x, const GbState* st, long long s, int lane,
                                                const GbTabs& Tb, double2* shF, double2* shM, float2* sh32) {
    constexpr bool tab = TAB;
    const long long nfree = st->nfree, bump = st->bump, kept_old = st->kept_old;
    const long long ci = ch.surv[s];
    ChildCtx c = child_ctx(par, ci, sp);
    if (tab) tab_dirty_groups(P, pool, Tb, c, ci, lane, shF, shM, sh32);
    const unsigned ns = (s < nfree) ? pool.freel[nfree - 1 - s] : (unsigned)(bump + (s - nfree));
    const int n = pool.n;
    View<double> X = view64(pool, par, c, sp);
    View<float> X32;
    if (pool.fp32) X32 = view32(pool, par, c, sp);
    bool narrow = true;
    for (int j = lane; j < n; j += 32) {
        iv64 x = X.get(j);
        pool.lo64[(size_t)ns * n + j] = x.lo;
        pool.hi64[(size_t)ns * n + j] = x.hi;
        if (pool.fp32) {
            iv32 y = X32.get(j);
            pool.lo32[(size_t)ns * n + j] = y.lo;
            pool.hi32[(size_t)ns * n + j] = y.hi;
        }
        if (!(__dsub_rn(x.hi, x.lo) < tol_x)) narrow = false;
    }
    narrow = __all_sync(0xffffffffu, narrow) && tol_x > 0.0;
    const int blk = c.info.z;
    MidView MX{X};
    iv64 R[TAB ? 1 : GB_MAX_TREGS];
    iv32 R32[TAB ? 1 : GB_MAX_TREGS];
    int slot_k = 0, ops = 0;
    for (int k = 0; k < P.n_sum; k++) {
        GbSum S = P.sums[k];
        int2 dr = P.dirty[blk * P.n_sum + k];
        for (int g = lane; g < S.ngroups; g += 32) {
            if (g >= dr.x && g < dr.y) continue;
            size_t src = (size_t)c.slot * pool.NG + S.group0 + g, dst = (size_t)ns * pool.NG + S.group0 + g;
            pool.gsum[dst] = pool.gsum[src];
            pool.gmid[dst] = pool.gmid[src];
            if (pool.fp32) pool.gsum32[dst] = pool.gsum32[src];
            for (int j = 0; pool.gsamp && j < pool.S; j++)
                pool.gsamp[((size_t)ns * pool.S + j) * pool.NG + S.group0 + g] =
                    pool.gsamp[((size_t)c.slot * pool.S + j) * pool.NG + S.group0 + g];
        }
        for (int g = dr.x; g < dr.y; g++, slot_k++) {
            if ((slot_k & 31) != lane) continue;
            size_t dst = (size_t)ns * pool.NG + S.group0 + g;
            iv64 a, b;
            if constexpr (TAB) {
                const int at = k * GB_TAB_MAX_DIRTY + (g - dr.x);
                a = iv64{shF[at].x, shF[at].y};
                b = iv64{shM[at].x, shM[at].y};
                if (pool.fp32) pool.gsum32[dst] = sh32[at];
            } else {
                a = group_sum<PR, double>(P, S, g, X, R, ops);
                b = group_sum<PR, double>(P, S, g, MX, R, ops);
                if (pool.fp32) {
                    iv32 f = group_sum<PR, float>(P, S, g, X32, R32, ops);
                    pool.gsum32[dst] = make_float2(f.lo, f.hi);
                }
            }
            pool.gsum[dst] = make_double2(a.lo, a.hi);
            pool.gmid[dst] = make_double2(b.lo, b.hi);
            if constexpr (!TAB)   // diagonal samples: paper mode runs on the interpreter only
                for (int j = 1; pool.gsamp && j <= pool.S; j++) {
                    const iv64 v = group_sum<PR, double>(P, S, g, SampleView{X, j, pool.S + 1}, R, ops);
                    pool.gsamp[((size_t)ns * pool.S + (j - 1)) * pool.NG + S.group0 + g] = make_double2(v.lo, v.hi);
                }
        }
    }
    if (!TAB && pool.gdp) {   // coordinate partials: the parent's, recomputed where the split reaches
        const int2 ab = d_affected(P, blk);
        const int a0 = ab.x * P.B, a1 = min(n, (ab.y + 1) * P.B);
        const double2* src = pool.gdp + (size_t)c.slot * P.n_sum * n;
        double2* dst = pool.gdp + (size_t)ns * P.n_sum * n;
        for (int k = 0; k < P.n_sum; k++)
            for (int j = lane; j < n; j += 32)
                if (j < a0 || j >= a1) dst[(size_t)k * n + j] = src[(size_t)k * n + j];
        iv64 RA[GB_MAX_TREGS];
        for (int b = ab.x + lane; b <= ab.y; b += 32) block_D(P, b, X, R, RA, dst, n, 0, ops);
    }
    if (lane == 0) {
        long long e = kept_old + s;
        En.flo[e] = ch.flo[ci];
        En.slot[e] = ns;
        En.cyc[e] = (int)((unsigned)c.info.w | (narrow ? GB_FINAL_BIT : 0u));
    }
}

// Survivor list of a generation with at most 2^16 children: one block
// does the count, the scan and the scatter.
__global__ void __launch_bounds__(1024) k_cc_small(GbChildren ch, GbGenConst G, GbState* st) {
    gb_grid_trigger();
    gb_grid_wait();
    if (st->halt) return;
    __shared__ int sw[32];
    const long long S = survivor_list_block(ch, st->nch, gb_key_value(st->gub_new_key), false, sw);
    if (threadIdx.x == 0) set_survivors(G, st, S);
}

// ---------------------------------------------------------------------------
// Block records: a box's row names one record per block, and a child shares
// all but the records of the blocks it changes with its parent, so a record
// is referenced by many boxes and is freed by a mark-and-sweep collection.
// It runs right after the pool partition, when the generation's new records
// might not fit (the partition's verdict: the most children a generation can
// keep, times the records a child writes, against the free and never-used
// records): stamp the records named by the boxes still alive (entries carried
// over and this generation's parents) with the collection's number, then
// list the unstamped ones in ascending order as the free list.  With one
// parent taken from its pool position (sel), the parent's slot is read there
// (the parent buffer is written by the table kernel, which may be running).
__global__ void k_gc_mark(GbPool pool, GbEntries En, GbParents par, const GbState* st, GbEntries E, int sel) {
    gb_grid_trigger();
    gb_grid_wait();
    if (st->halt || !st->gc) return;
    const long long nbox = st->kept_old + st->parents, nb = pool.nb;
    const unsigned sel_slot = sel ? E.slot[st->sel_pos] : 0u;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nbox * nb;
         i += (long long)gridDim.x * blockDim.x) {
        const long long q = i / nb, b = i - q * nb;
        const unsigned slot = q < st->kept_old ? En.slot[q] : (sel ? sel_slot : par.slot[q - st->kept_old]);
        pool.rmark[pool.rid[(size_t)slot * nb + b]] = (unsigned)(st->rec_gc + 1);
    }
}

__device__ __forceinline__ bool rec_free(const GbPool& pool, long long id, long long used, unsigned epoch) {
    return id < used && pool.rmark[id] != epoch;
}

__global__ void k_gc_count(GbPool pool, const GbState* st, int* tile_cnt) {
    gb_grid_trigger();
    gb_grid_wait();
    if (st->halt || !st->gc) return;
    __shared__ int sw[PT / 32 + 1];
    const long long used = st->rec_bump, nt = ntiles_of(used);
    const unsigned epoch = (unsigned)(st->rec_gc + 1);
    for (long long tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        int acc = 0, tot;
        for (int r = 0; r < GB_TILE / PT; r++) {
            block_prefix<PT>(rec_free(pool, tile * GB_TILE + r * PT + threadIdx.x, used, epoch), sw, &tot);
            acc += tot;
        }
        if (threadIdx.x == 0) tile_cnt[tile] = acc;
    }
}

__global__ void k_gc_scatter(GbPool pool, const GbState* st, const int* tile_off) {
    gb_grid_trigger();
    gb_grid_wait();
    if (st->halt || !st->gc) return;
    __shared__ int sw[PT / 32 + 1];
    const long long used = st->rec_bump, nt = ntiles_of(used);
    const unsigned epoch = (unsigned)(st->rec_gc + 1);
    for (long long tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        long long o = tile_off[tile];
        for (int r = 0; r < GB_TILE / PT; r++) {
            const long long id = tile * GB_TILE + r * PT + threadIdx.x;
            const bool f = rec_free(pool, id, used, epoch);
            int tot;
            const int rk = block_prefix<PT>(f, sw, &tot);
            if (f) pool.rfree[o + rk] = (unsigned)id;
            o += tot;
        }
    }
}

// Block records: survivor s takes new records s * nrec + t (t = 0 .. nrec-1,
// from the free list, then never-used ones) for blocks blk - t, the blocks
// whose owned groups can touch the split block blk; its row is its parent's
// with those entries replaced.  A new record holds the child's coordinates of
// its block and the cached sums of the groups it owns (groups of the dirty
// ranges recomputed, the others copied from the parent's record).
template <bool PR, bool TAB>
__device__ __forceinline__ void materialize_rec(const GbProg& P, const GbPool& pool, const GbParents& par,
                                                const GbChildren& ch, const GbSplit& sp, const GbEntries& En,
                                                double tol_x, const GbState* st, long long s, int lane,
                                                const GbTabs& Tb, double2* shF, double2* shM, float2* sh32) {
    constexpr bool tab = TAB;
    const long long nfree = st->nfree, bump = st->bump, kept_old = st->kept_old;
    const long long rnf = st->rec_nfree, rbump = st->rec_bump;
    const long long ci = ch.surv[s];
    const ChildCtx c = child_ctx(par, ci, sp);
    if (tab) tab_dirty_groups(P, pool, Tb, c, ci, lane, shF, shM, sh32);
    const unsigned ns = (s < nfree) ? pool.freel[nfree - 1 - s] : (unsigned)(bump + (s - nfree));
    const int n = pool.n, nb = pool.nb, B = pool.B, GPB = pool.GPB, nrec = pool.nrec;
    const int blk = c.info.z;
    const unsigned* prow = pool.rid + (size_t)c.slot * nb;
    unsigned* crow = pool.rid + (size_t)ns * nb;
    for (int b = lane; b < nb; b += 32) {
        const int t = blk - b;
        unsigned id = prow[b];
        if (t >= 0 && t < nrec) {
            const long long q = s * nrec + t;
            id = q < rnf ? pool.rfree[rnf - 1 - q] : (unsigned)(rbump + (q - rnf));
        }
        crow[b] = id;
    }
    __syncwarp();
    const View<double> X = view64(pool, par, c, sp);
    View<float> X32;
    if (pool.fp32) X32 = view32(pool, par, c, sp);
    int wide_delta = 0;
    // the child's coordinates of each new record: the parent's record of that
    // block, with the split coordinates' pieces; each lane loads its batch of
    // coordinates before storing any (the stores go to the arrays the loads
    // read, so they would otherwise wait one memory round trip each)
    constexpr int BATCH = 4;
    const size_t bo = (size_t)c.p * sp.dmax * (sp.m + 1);
    for (int t = 0; t < nrec && blk - t >= 0; t++) {
        const int b = blk - t, j0 = b * B, j1 = min(n, j0 + B);
        const size_t o = (size_t)crow[b] * B, src = (size_t)prow[b] * B;
        bool wide = false;
        for (int jb = j0; jb < j1; jb += 32 * BATCH) {
            double xl[BATCH], xh[BATCH];
            float yl[BATCH], yh[BATCH];
#pragma unroll
            for (int u = 0; u < BATCH; u++) {
                const int j = jb + u * 32 + lane;
                if (j >= j1) continue;
                const unsigned k = (unsigned)(j - c.info.x);
                if (k < (unsigned)c.info.y) {   // a split coordinate: its piece's boundaries
                    const int dig = (c.r >> (k * sp.mshift)) & ((1 << sp.mshift) - 1);
                    const size_t at = bo + (size_t)k * (sp.m + 1) + dig;
                    xl[u] = par.bnd[at];
                    xh[u] = par.bnd[at + 1];
                    if (pool.fp32) {
                        yl[u] = par.bnd_rd[at];
                        yh[u] = par.bnd_ru[at + 1];
                    }
                } else {
                    xl[u] = pool.rlo[src + (j - j0)];
                    xh[u] = pool.rhi[src + (j - j0)];
                    if (pool.fp32) {
                        yl[u] = pool.rlo32[src + (j - j0)];
                        yh[u] = pool.rhi32[src + (j - j0)];
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < BATCH; u++) {
                const int j = jb + u * 32 + lane;
                if (j >= j1) continue;
                pool.rlo[o + (j - j0)] = xl[u];
                pool.rhi[o + (j - j0)] = xh[u];
                if (pool.fp32) {
                    pool.rlo32[o + (j - j0)] = yl[u];
                    pool.rhi32[o + (j - j0)] = yh[u];
                }
                if (!(__dsub_rn(xh[u], xl[u]) < tol_x)) wide = true;
            }
        }
        wide = __any_sync(0xffffffffu, wide);
        if (lane == 0) {
            pool.rwide[crow[b]] = wide ? 1 : 0;
            wide_delta += (wide ? 1 : 0) - (int)pool.rwide[prow[b]];
        }
    }
    const MidView MX{X};
    iv64 R[TAB ? 1 : GB_MAX_TREGS];
    iv32 R32[TAB ? 1 : GB_MAX_TREGS];
    int ops = 0;
    for (int it = lane; it < nrec * GPB; it += 32) {
        const int t = it / GPB, o = it - t * GPB, b = blk - t;
        if (b < 0) continue;
        const int g = P.owned[(size_t)b * GPB + o];
        if (g < 0) continue;
        int k = 0;
        while (k + 1 < P.n_sum && P.sums[k + 1].group0 <= g) k++;
        const GbSum S = P.sums[k];
        const int gl = g - S.group0;
        const int2 dr = P.dirty[blk * P.n_sum + k];
        const size_t dst = (size_t)crow[b] * GPB + o, src = (size_t)prow[b] * GPB + o;
        const size_t sstep = (size_t)pool.R * GPB;   // sample j's sums: rgsamp + (j - 1) * sstep
        if (gl < dr.x || gl >= dr.y) {
            pool.rgsum[dst] = pool.rgsum[src];
            pool.rgmid[dst] = pool.rgmid[src];
            if (pool.fp32) pool.rgsum32[dst] = pool.rgsum32[src];
            for (int j = 0; pool.rgsamp && j < pool.S; j++) pool.rgsamp[j * sstep + dst] = pool.rgsamp[j * sstep + src];
            continue;
        }
        if constexpr (!TAB)   // diagonal samples: paper mode runs on the interpreter only
            for (int j = 1; pool.rgsamp && j <= pool.S; j++) {
                const iv64 v = group_sum<PR, double>(P, S, gl, SampleView{X, j, pool.S + 1}, R, ops);
                pool.rgsamp[(j - 1) * sstep + dst] = make_double2(v.lo, v.hi);
            }
        iv64 a, m;
        if constexpr (TAB) {
            const int at = k * GB_TAB_MAX_DIRTY + (gl - dr.x);
            a = iv64{shF[at].x, shF[at].y};
            m = iv64{shM[at].x, shM[at].y};
            if (pool.fp32) pool.rgsum32[dst] = sh32[at];
        } else {
            a = group_sum<PR, double>(P, S, gl, X, R, ops);
            m = group_sum<PR, double>(P, S, gl, MX, R, ops);
            if (pool.fp32) {
                const iv32 f = group_sum<PR, float>(P, S, gl, X32, R32, ops);
                pool.rgsum32[dst] = make_float2(f.lo, f.hi);
            }
        }
        pool.rgsum[dst] = make_double2(a.lo, a.hi);
        pool.rgmid[dst] = make_double2(m.lo, m.hi);
    }
    if (!TAB && pool.rgdp) {   // coordinate partials of each new record's block (templates within one coordinate)
        iv64 RA[GB_MAX_TREGS];
        for (int t = lane; t < nrec && blk - t >= 0; t += 32) {
            const int b = blk - t;
            block_D(P, b, X, R, RA, pool.rgdp + (size_t)crow[b] * P.n_sum * B, B, b * B, ops);
        }
    }
    if (lane == 0) {
        const int w = pool.swide[c.slot] + wide_delta;
        pool.swide[ns] = w;
        const bool narrow = tol_x > 0.0 && w == 0;
        const long long e = kept_old + s;
        En.flo[e] = ch.flo[ci];
        En.slot[e] = ns;
        En.cyc[e] = (int)((unsigned)c.info.w | (narrow ? GB_FINAL_BIT : 0u));
    }
}

// The survivors into the pool, one warp per survivor.  With the end of the
// generation fused (K = 1; `pkey` non-null): each block also leaves the
// smallest key of its new entries that can be selected (not final) and its
// last position after the npart pairs of the partition, and the last block
// to finish ends the generation: the parent's slot back to the free list (on
// overflow the parent back into the pool), the counters rolled forward, and
// the next selection.  For K = 1 the smallest selectable key of the new pool
// is all the selection needs: its entry is the next parent when it is below
// the new incumbent's cut-off threshold, and if it is not, no entry is.
template <bool PR, bool RECS, bool TAB>
__global__ void __launch_bounds__(128) k_materialize(GbProg P, GbPool pool, GbParents par, GbChildren ch,
                                                     GbSplit sp, GbEntries En, double tol_x, GbState* st,
                                                     GbTabs Tb, GbGenConst G, int npart, unsigned long long* pkey,
                                                     long long* ppos) {
    gb_grid_trigger();
    gb_grid_wait();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __shared__ double2 shF[4][GB_SHG], shM[4][GB_SHG];
    __shared__ float2 sh32[4][GB_SHG];
    __shared__ unsigned long long s_bk[4];
    __shared__ long long s_bq[4];
    __shared__ bool s_last;
    if (st->halt) return;
    const long long kept = st->overflow ? 0 : st->kept;
    const long long kept_old = st->kept_old;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    unsigned long long bk = ~0ull;
    long long bq = -1;
    for (long long s = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; s < kept; s += nwarps) {
        if constexpr (RECS)
            materialize_rec<PR, TAB>(P, pool, par, ch, sp, En, tol_x, st, s, lane, Tb, shF[w], shM[w], sh32[w]);
        else
            materialize_one<PR, TAB>(P, pool, par, ch, sp, En, tol_x, st, s, lane, Tb, shF[w], shM[w], sh32[w]);
        __syncwarp();
        if (pkey && lane == 0) {   // the entry lane 0 has just written
            const long long e = kept_old + s;
            const int cy = En.cyc[e];
            if (!((unsigned)cy & GB_FINAL_BIT)) better_key(bk, bq, gb_order_key(En.flo[e]), e);
        }
    }
    if (!pkey) return;
    block_best(bk, bq, s_bk, s_bq);
    if (threadIdx.x == 0) {
        pkey[npart + blockIdx.x] = bk;
        ppos[npart + blockIdx.x] = bq;
    }
    if (!arrive_last(&st->stats_done, gridDim.x, &s_last)) return;
    free_parents(par, pool, En, st, threadIdx.x, blockDim.x);
    unsigned long long mk;
    long long mq;
    combine_pairs(pkey, ppos, npart + (int)gridDim.x, mk, mq, s_bk, s_bq);   // (synchronises the block)
    if (threadIdx.x != 0) return;
    finish_counters(G, st);
    const bool active = mq >= 0 && gb_key_value(mk) < thr_of(gb_key_value(st->gub_key), G.tol_f);
    open_generation(G, st, active ? 1 : 0, mk, mq);
}

// ---------------------------------------------------------------------------
// Output: entries with LB <= GUB (stable), gathered into rows; GLB = min LB.
__global__ void k_out_count(GbEntries E, long long count, double gub, int* tile_cnt, GbState* st) {
    __shared__ int sw[PT / 32 + 1];
    const long long base = (long long)blockIdx.x * GB_TILE;
    int acc = 0, tot;
    unsigned long long kmin = ~0ull;
    for (int r = 0; r < GB_TILE / PT; r++) {
        long long q = base + r * PT + threadIdx.x;
        bool f = q < count && !(E.flo[q] > gub);
        if (f) {
            unsigned long long k = gb_order_key(E.flo[q]);
            kmin = k < kmin ? k : kmin;
        }
        block_prefix<PT>(f, sw, &tot);
        acc += tot;
    }
    for (int o = 16; o; o >>= 1) {
        unsigned long long other = __shfl_down_sync(0xffffffffu, kmin, o);
        kmin = other < kmin ? other : kmin;
    }
    if ((threadIdx.x & 31) == 0 && kmin != ~0ull) atomicMin(&st->glb_key, kmin);
    if (threadIdx.x == 0) tile_cnt[blockIdx.x] = acc;
}

__global__ void k_out_scatter(GbEntries E, long long count, double gub, const int* tile_off, unsigned* list) {
    __shared__ int sw[PT / 32 + 1];
    const long long base = (long long)blockIdx.x * GB_TILE;
    long long o = tile_off[blockIdx.x];
    for (int r = 0; r < GB_TILE / PT; r++) {
        long long q = base + r * PT + threadIdx.x;
        bool f = q < count && !(E.flo[q] > gub);
        int tot;
        int rk = block_prefix<PT>(f, sw, &tot);
        if (f) list[o + rk] = (unsigned)q;
        o += tot;
    }
}

__global__ void k_out_gather(GbEntries E, const unsigned* list, const GbState* st, GbPool pool, double* out_lo,
                             double* out_hi, double* out_flo) {
    const int lane = threadIdx.x & 31;
    const long long b = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    if (b >= st->kept) return;
    unsigned q = list[b];
    unsigned slot = E.slot[q];
    const int n = pool.n;
    const View<double> X = box_view64(pool, slot);
    for (int j = lane; j < n; j += 32) {
        const iv64 x = X.get(j);
        out_lo[(size_t)b * n + j] = x.lo;
        out_hi[(size_t)b * n + j] = x.hi;
    }
    if (lane == 0) out_flo[b] = E.flo[q];
}

// ---------------------------------------------------------------------------
// Parity hook: full evaluation of given boxes.
// ---------------------------------------------------------------------------
// Checkpoint and resume of the pool (the list L of section 3.1).
// Every pool entry in pool order: its box, lower bound and cycling word.
__global__ void k_snap_gather(GbEntries E, long long count, GbPool pool, double* out_lo, double* out_hi,
                              double* out_flo, int* out_cyc) {
    const int lane = threadIdx.x & 31;
    const long long q = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    if (q >= count) return;
    const unsigned slot = E.slot[q];
    const int n = pool.n;
    const View<double> X = box_view64(pool, slot);
    for (int j = lane; j < n; j += 32) {
        const iv64 x = X.get(j);
        out_lo[(size_t)q * n + j] = x.lo;
        out_hi[(size_t)q * n + j] = x.hi;
    }
    if (lane == 0) {
        out_flo[q] = E.flo[q];
        out_cyc[q] = E.cyc[q];
    }
}

// Resume (dense rows): box q goes to slot q and entry q; its FP32 shadow is
// the outward float of its bounds (as the root's and every split boundary's
// are), its group caches (F, midpoint, FP32, samples) and coordinate
// partials are recomputed in full, so a child of it reads the same cached
// values as a child of the original box.  One warp per box.
template <bool PR>
__global__ void __launch_bounds__(128) k_resume_boxes(GbProg P, GbPool pool, GbEntries E, long long count,
                                                      const double* lo, const double* hi, const double* flo,
                                                      const int* cyc) {
    const int lane = threadIdx.x & 31;
    const long long q = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    if (q >= count) return;
    const int n = P.n;
    const unsigned slot = (unsigned)q;
    for (int j = lane; j < n; j += 32) {
        const double a = lo[(size_t)q * n + j], b = hi[(size_t)q * n + j];
        pool.lo64[(size_t)slot * n + j] = a;
        pool.hi64[(size_t)slot * n + j] = b;
        if (pool.fp32) {
            pool.lo32[(size_t)slot * n + j] = __double2float_rd(a);
            pool.hi32[(size_t)slot * n + j] = __double2float_ru(b);
        }
    }
    __syncwarp();
    const View<double> X = box_view64(pool, slot);
    const MidView MX{X};
    View<float> X32;
    if (pool.fp32) X32 = box_view32(pool, slot);
    iv64 R[GB_MAX_TREGS];
    iv32 R32[GB_MAX_TREGS];
    int ops = 0;
    for (int k = 0; k < P.n_sum; k++) {
        const GbSum S = P.sums[k];
        for (int g = lane; g < S.ngroups; g += 32) {
            const size_t at = (size_t)slot * pool.NG + S.group0 + g;
            const iv64 a = group_sum<PR, double>(P, S, g, X, R, ops);
            const iv64 b = group_sum<PR, double>(P, S, g, MX, R, ops);
            pool.gsum[at] = make_double2(a.lo, a.hi);
            pool.gmid[at] = make_double2(b.lo, b.hi);
            if (pool.fp32) {
                const iv32 c = group_sum<PR, float>(P, S, g, X32, R32, ops);
                pool.gsum32[at] = make_float2(c.lo, c.hi);
            }
            for (int j = 1; pool.gsamp && j <= pool.S; j++) {
                const iv64 v = group_sum<PR, double>(P, S, g, SampleView{X, j, pool.S + 1}, R, ops);
                pool.gsamp[((size_t)slot * pool.S + (j - 1)) * pool.NG + S.group0 + g] = make_double2(v.lo, v.hi);
            }
        }
    }
    if (pool.gdp) {
        iv64 RA[GB_MAX_TREGS];
        for (int b = lane; b < P.nb; b += 32)
            block_D(P, b, X, R, RA, pool.gdp + (size_t)slot * P.n_sum * n, n, 0, ops);
    }
    if (lane == 0) {
        E.flo[q] = flo[q];
        E.slot[q] = slot;
        E.cyc[q] = cyc[q];
    }
}

// The device state of a resumed solve: `count` entries, incumbent gub.
__global__ void k_resume_state(long long count, double gub, GbState* st) {
    GbState s0 = {};
    s0.pool = count;
    s0.nfree = 0;
    s0.bump = count;
    s0.cap = st->cap;
    s0.gub_key = gb_order_key(gub);
    s0.gub_new_key = s0.gub_key;
    s0.sel_T = ~0ull;
    s0.min_key = ~0ull;
    *st = s0;
}

__global__ void k_to_f32(const double* lo, const double* hi, float* lo32, float* hi32, long long count) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= count) return;
    lo32[i] = __double2float_rd(lo[i]);
    hi32[i] = __double2float_ru(hi[i]);
}

template <bool PR>
__global__ void __launch_bounds__(128) k_eval_boxes(GbProg P, const double* lo, const double* hi,
                                                    const float* lo32, const float* hi32, long long nbox,
                                                    int blk, int fp32, double* Fo, double* Fmo, double* Go,
                                                    int* mono) {
    long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    const int n = P.n;
    View<double> X{lo + (size_t)b * n, hi + (size_t)b * n, nullptr, nullptr, 0, 0, 1, 2, 0u};
    MidView MX{X};
    iv64 R[GB_MAX_TREGS], O[GB_MAX_OREGS], sums[GB_MAX_ISUM];
    int ops = 0;
    sum_values<PR, double>(P, blk, MX, (const CacheRef<double2>*)nullptr, R, sums, ops);
    iv64 Fm = outer_fwd<double>(P, MX, sums, O, ops);
    Fmo[2 * b] = Fm.lo;
    Fmo[2 * b + 1] = Fm.hi;
    if (!fp32) {
        iv64 RA[GB_MAX_TREGS], OA[GB_MAX_OREGS];
        sum_values<PR, double>(P, blk, X, (const CacheRef<double2>*)nullptr, R, sums, ops);
        iv64 F = outer_fwd<double>(P, X, sums, O, ops);
        Fo[2 * b] = F.lo;
        Fo[2 * b + 1] = F.hi;
        if (blk >= 0) {
            bool m = block_mono<PR, double>(P, blk, X, X, O, OA, R, RA, Go + (size_t)b * P.B * 2,
                                        (const CacheRef<double2>*)nullptr, -1, ops);
            mono[b] = m ? 1 : 0;
        }
    } else {
        View<float> X32{lo32 + (size_t)b * n, hi32 + (size_t)b * n, nullptr, nullptr, 0, 0, 1, 2, 0u};
        iv32 R32[GB_MAX_TREGS], RA32[GB_MAX_TREGS], O32[GB_MAX_OREGS], OA32[GB_MAX_OREGS], s32[GB_MAX_ISUM];
        sum_values<PR, float>(P, blk, X32, (const CacheRef<float2>*)nullptr, R32, s32, ops);
        iv32 F = outer_fwd<float>(P, X32, s32, O32, ops);
        Fo[2 * b] = F.lo;
        Fo[2 * b + 1] = F.hi;
        if (blk >= 0) {
            bool m = block_mono<PR, float>(P, blk, X32, X, O32, OA32, R32, RA32, Go + (size_t)b * P.B * 2,
                                       (const CacheRef<float2>*)nullptr, -1, ops);
            mono[b] = m ? 1 : 0;
        }
    }
}

// ---------------------------------------------------------------------------
// Directed-rounding throughput probe: 8 independent chains per thread,
// 4 additions rounded down and 4 multiplications rounded up per iteration.
template <typename T>
__global__ void __launch_bounds__(256) k_peak(int iters, T seed, T inc, T mul, T* sink) {
    T a0 = seed + (T)threadIdx.x, a1 = a0 + (T)1, a2 = a0 + (T)2, a3 = a0 + (T)3;
    T m0 = (T)1 + (T)threadIdx.x * (T)1e-7, m1 = m0, m2 = m0, m3 = m0;
    for (int i = 0; i < iters; i++) {
        a0 = add_rd(a0, inc); a1 = add_rd(a1, inc); a2 = add_rd(a2, inc); a3 = add_rd(a3, inc);
        m0 = mul_ru(m0, mul); m1 = mul_ru(m1, mul); m2 = mul_ru(m2, mul); m3 = mul_ru(m3, mul);
    }
    T s = a0 + a1 + a2 + a3 + m0 + m1 + m2 + m3;
    if (s == (T)-1) sink[threadIdx.x] = s;   // never taken; keeps the chains live
}

inline unsigned grid_for(long long items, int per_block) {
    long long g = (items + per_block - 1) / per_block;
    return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

// ===========================================================================
// launch wrappers (each adds the number of kernels it launched to the
// calling thread's counter)
thread_local long long gb_launch_count = 0;

long long gb_launches_so_far() { return gb_launch_count; }

static thread_local bool t_pdl_off = false;

void gb_pdl_thread(bool on) { t_pdl_off = !on; }

bool gb_pdl_enabled() {
    static int on = -1;   // read once
    int v = __atomic_load_n(&on, __ATOMIC_RELAXED);
    if (v < 0) {
        const char* e = std::getenv("GB_PDL");
        v = (e && e[0] == '1') ? 1 : 0;
        __atomic_store_n(&on, v, __ATOMIC_RELAXED);
    }
    return v != 0 && !t_pdl_off;
}

int gb_sm_count() {
    static int sms[64];   // per device ordinal, 0 until queried
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    int v = __atomic_load_n(&sms[dev], __ATOMIC_RELAXED);
    if (v <= 0) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) return 152;
        __atomic_store_n(&sms[dev], v, __ATOMIC_RELAXED);
    }
    return v;
}
cudaError_t gb_launch_root_init(const GbProg& P, const GbPool& pool, const GbEntries& E, double tol_x,
                                GbState* st, cudaStream_t s) {
    gb_launch_count++;
    if (P.any_prod) k_root_init<true><<<1, 256, 0, s>>>(P, pool, E, tol_x, st);
    else k_root_init<false><<<1, 256, 0, s>>>(P, pool, E, tol_x, st);
    return cudaGetLastError();
}

cudaError_t gb_launch_snapshot(const GbEntries& E, long long count, const GbPool& pool, double* lo, double* hi,
                               double* flo, int* cyc, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    gb_launch_count++;
    k_snap_gather<<<grid_for(count * 32, 128), 128, 0, s>>>(E, count, pool, lo, hi, flo, cyc);
    return cudaGetLastError();
}

cudaError_t gb_launch_resume(const GbProg& P, const GbPool& pool, const GbEntries& E, long long count,
                             const double* lo, const double* hi, const double* flo, const int* cyc, double gub,
                             GbState* st, cudaStream_t s) {
    if (count > 0) {
        gb_launch_count++;
        if (P.any_prod)
            k_resume_boxes<true><<<grid_for(count * 32, 128), 128, 0, s>>>(P, pool, E, count, lo, hi, flo, cyc);
        else
            k_resume_boxes<false><<<grid_for(count * 32, 128), 128, 0, s>>>(P, pool, E, count, lo, hi, flo, cyc);
    }
    gb_launch_count++;
    k_resume_state<<<1, 1, 0, s>>>(count, gub, st);
    return cudaGetLastError();
}

cudaError_t gb_launch_stats(const GbEntries& E, const GbGenConst& G, long long cap, const GbScan& sc, GbState* st,
                            cudaStream_t s, const GbParents* par, const GbPool* pool) {
    unsigned g = grid_for(cap, 256);
    if (g > gb_sm_count() * 8) g = gb_sm_count() * 8;
    if (g > (unsigned)GB_STAT_BLOCKS) g = GB_STAT_BLOCKS;
    gb_launch_count++;
    return gb_launch_ex(k_stats, g, 256, 0, s, par != nullptr, E, G, st, sc.stat_key, sc.stat_pos,
                        par ? *par : GbParents{}, pool ? *pool : GbPool{}, par ? 1 : 0);
}

cudaError_t gb_launch_generation(const GbProg& P, const GbPool& pool, const GbEntries& E, const GbEntries& E_new,
                                 const GbParents& par, const GbChildren& ch, const GbSplit& sp, const GbScan& sc,
                                 const GbTabs* tabs, const GbGenConst& G, long long cap, long long Cmax,
                                 GbState* st, cudaStream_t s, cudaEvent_t* ev, long long* nlaunch, int part,
                                 const GbFork* fork) {
    long long n0 = gb_launch_count;
    cudaError_t e;
    const unsigned gpool = (unsigned)std::min<long long>(grid_for(cap, 256), gb_sm_count() * 8);
    const unsigned gtile_pool = (unsigned)std::min<long long>(grid_for(cap, GB_TILE), gb_sm_count() * 8);
    const unsigned gtile_ch = (unsigned)std::min<long long>(grid_for(Cmax, GB_TILE), gb_sm_count() * 8);
    const unsigned gch = (unsigned)std::min<long long>(grid_for(Cmax, 128), gb_sm_count() * 32);
    const unsigned gmat_max = (unsigned)std::min<long long>(grid_for(Cmax * 32, 128), gb_sm_count() * 16);
    // K = 1: the partition and k_materialize leave per-block (key, position)
    // pairs and k_materialize's last block ends the generation
    const bool fuse_end = G.K == 1 && gtile_pool <= (unsigned)GB_STAT_BLOCKS && 1 + gmat_max <= (unsigned)GB_STAT_BLOCKS;
    bool cc_done = false;   // the survivor list came with the child kernel
    // part 0: the whole generation; 1: up to the child evaluation; 2: after it
    if (part == 2) goto after_eval;
    {
    // (the selection was chosen at the end of the last generation)
    if (G.K > 1) {
        for (int pass = 0; pass < 4; pass++) {
            gb_launch_count += 2;
            k_radix_hist<<<gpool, 256, 0, s>>>(E, G, pass, st, sc.hist);
            k_radix_pick<<<1, 1024, 0, s>>>(pass, st, sc.hist);
        }
    }
    // K = 1 with term tables: the parent is the pool entry the last k_stats
    // found, so its tables need nothing from the partition and run beside it
    // (on the fork stream when there is one), joined before the children
    const bool sel_tabs = tabs && G.K == 1;
    cudaStream_t ts = s;
    if (sel_tabs && fork) {
        if ((e = cudaEventRecord(fork->fork, s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(fork->s2, fork->fork, 0)) != cudaSuccess) return e;
        ts = fork->s2;
    }
    auto tables = [&]() -> cudaError_t {
        cudaError_t et;
        // the evaluation window (ev[0] .. ev[1]): per-parent tables and every child kernel
        if (ev && part == 0) cudaEventRecord(ev[0], ts);
        gb_launch_count++;
        if ((et = gb_launch_ptab(P, pool, par, *tabs, G.K, sp, st, ts, sel_tabs ? &E : nullptr)) != cudaSuccess)
            return et;
        gb_launch_count++;
        if ((et = gb_launch_ptab_d(P, pool, par, *tabs, G.K, P.B, st, ts, sel_tabs)) != cudaSuccess) return et;
        if (tabs->cs64) {
            gb_launch_count++;
            if ((et = gb_launch_child_sums(P, pool, par, *tabs, sp, Cmax, G.fp32, st, ts, sel_tabs)) != cudaSuccess)
                return et;
        }
        return cudaSuccess;
    };
    if (sel_tabs && (e = tables()) != cudaSuccess) return e;
    gb_launch_count++;
    // beside the tables the partition keeps to two blocks per SM (its blocks
    // take tiles by ticket, so fewer blocks only take more tiles each) and
    // leaves room for the table kernels' blocks
    const unsigned gpart = ts != s ? std::min<unsigned>(gtile_pool, (unsigned)gb_sm_count() * 2) : gtile_pool;
    if ((e = gb_launch_ex(k_part_1p, gpart, PT, 0, s, true, E, G, st, sc.tile_cnt, sc.tile_off, sc.max_tiles,
                          sc.tile_flag, E_new, par, pool.freel, sel_tabs ? 1 : 0, fuse_end ? sc.stat_key : nullptr,
                          fuse_end ? sc.stat_pos : nullptr)) != cudaSuccess)
        return e;
    if (pool.recs) {   // the record collection, when the partition asked for it
        // Launched without the early start: their blocks would otherwise sit
        // on the SMs, waiting for the partition, in the way of the tables'
        // blocks; two blocks per SM, as they mostly return at once.
        const unsigned ggc = (unsigned)gb_sm_count() * 2;
        const unsigned grec = (unsigned)std::min<long long>(grid_for(pool.R, GB_TILE), ggc);
        gb_launch_count += 4;
        if ((e = gb_launch_ex(k_gc_mark, ggc, 256, 0, s, false, pool, E_new, par, st, E, sel_tabs ? 1 : 0)) !=
                cudaSuccess ||
            (e = gb_launch_ex(k_gc_count, grec, PT, 0, s, false, pool, st, sc.tile_cnt)) != cudaSuccess ||
            (e = gb_launch_ex(k_scan_tiles, 1, 1024, 0, s, false, 1, sc.tile_cnt, sc.tile_off, sc.max_tiles, 4, 0LL,
                              G, st)) != cudaSuccess ||
            (e = gb_launch_ex(k_gc_scatter, grec, PT, 0, s, false, pool, st, sc.tile_off)) != cudaSuccess)
            return e;
    }
    if (!tabs) {   // with term tables k_ptab splits the parents itself
        gb_launch_count++;
        k_prep<<<grid_for(G.K * (long long)sp.dmax, 128), 128, 0, s>>>(P, pool, par, sp, st);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (ev && part == 0) cudaEventRecord(ev[0], s);
    } else if (!sel_tabs) {
        if ((e = tables()) != cudaSuccess) return e;
    }
    if (ts != s) {
        if ((e = cudaEventRecord(fork->join, ts)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(s, fork->join, 0)) != cudaSuccess) return e;
    }
    if (part == 1) {   // up to the child evaluation (a fused launch over many problems follows)
        if (nlaunch) *nlaunch = gb_launch_count - n0;
        return cudaGetLastError();
    }
    const bool fused = G.fp32 && tabs && tabs->warp;
    if (fused) {
        // FP32 prefilter and FP64 evaluation in one warp-per-child kernel
        if (ev) cudaEventRecord(ev[2], s), cudaEventRecord(ev[3], s);
        gb_launch_count++;
        cc_done = Cmax <= 64LL * 128;   // (at most 64 children per thread of the last block)
        if ((e = gb_launch_eval3264_tabw(P, pool, par, *tabs, ch, Cmax, sp, st, s, cc_done ? &G : nullptr)) !=
            cudaSuccess)
            return e;
        if (ev) cudaEventRecord(ev[1], s);
    } else {
        if (G.fp32) {
            if (ev) cudaEventRecord(ev[2], s);
            if (tabs) {
                gb_launch_count++;
                if ((e = gb_launch_eval32_tab(P, pool, par, *tabs, ch, Cmax, sp, st, s)) != cudaSuccess) return e;
            } else {
                gb_launch_count++;
                if (P.any_prod) k_eval32<true><<<gch, 128, 0, s>>>(P, pool, par, ch, sp, st);
                else k_eval32<false><<<gch, 128, 0, s>>>(P, pool, par, ch, sp, st);
            }
            if (ev) cudaEventRecord(ev[3], s);
            gb_launch_count += 3;
            k_cc_count<<<gtile_ch, PT, 0, s>>>(ch, 0, st, sc.tile_cnt);
            k_scan_tiles<<<1, 1024, 0, s>>>(1, sc.tile_cnt, sc.tile_off, sc.max_tiles, 1, 0, G, st);
            k_cc_scatter<<<gtile_ch, PT, 0, s>>>(ch, 0, st, sc.tile_off, ch.list32);
        }
        if (tabs) {
            gb_launch_count++;
            if ((e = gb_launch_eval64_tab(P, pool, par, *tabs, ch, Cmax, sp, G.fp32 != 0, st, s)) != cudaSuccess)
                return e;
        } else {
            gb_launch_count++;
            if (P.any_prod) k_eval64<true><<<gch, 128, 0, s>>>(P, pool, par, ch, sp, G.fp32, st);
            else k_eval64<false><<<gch, 128, 0, s>>>(P, pool, par, ch, sp, G.fp32, st);
        }
        if (ev) cudaEventRecord(ev[1], s);
    }
    }
after_eval:
    if (cc_done) {
        // (listed by the child kernel's last block)
    } else if (Cmax <= (1LL << 16)) {
        gb_launch_count++;
        if ((e = gb_launch_ex(k_cc_small, 1, 1024, 0, s, true, ch, G, st)) != cudaSuccess) return e;
    } else {
        gb_launch_count += 3;
        if ((e = gb_launch_ex(k_cc_count, gtile_ch, PT, 0, s, true, ch, 1, st, sc.tile_cnt)) != cudaSuccess ||
            (e = gb_launch_ex(k_scan_tiles, 1, 1024, 0, s, true, 1, sc.tile_cnt, sc.tile_off, sc.max_tiles, 2, 0LL,
                              G, st)) != cudaSuccess ||
            (e = gb_launch_ex(k_cc_scatter, gtile_ch, PT, 0, s, true, ch, 1, st, sc.tile_off, ch.surv)) != cudaSuccess)
            return e;
    }
    GbTabs Tb{};
    if (tabs) Tb = *tabs;
    gb_launch_count++;
    const unsigned gmat = gmat_max;
    // K = 1: the generation ends in k_materialize's last block (no k_stats pass)
    unsigned long long* pk = fuse_end ? sc.stat_key : nullptr;
    long long* pq = fuse_end ? sc.stat_pos : nullptr;
    const int np = 1;   // the partition's combined pair
#define GB_MAT(PR, RECS, TAB)                                                                                      \
    e = gb_launch_ex(k_materialize<PR, RECS, TAB>, gmat, 128, 0, s, true, P, pool, par, ch, sp, E_new, G.tol_x,   \
                     st, Tb, G, np, pk, pq)
    // products never use term tables
    if (P.any_prod) {
        if (pool.recs) GB_MAT(true, true, false);
        else GB_MAT(true, false, false);
    } else if (tabs) {
        if (pool.recs) GB_MAT(false, true, true);
        else GB_MAT(false, false, true);
    } else {
        if (pool.recs) GB_MAT(false, true, false);
        else GB_MAT(false, false, false);
    }
#undef GB_MAT
    if (e != cudaSuccess) return e;
    // otherwise the end of the generation (parents freed, counters) and the
    // statistics of the new pool, which start the next generation
    if (!fuse_end && (e = gb_launch_stats(E_new, G, cap, sc, st, s, &par, &pool)) != cudaSuccess) return e;
    if (nlaunch) *nlaunch = gb_launch_count - n0;
    return cudaGetLastError();
}

cudaError_t gb_launch_output(const GbEntries& E, long long count, const GbPool& pool, double gub, unsigned* list,
                             double* out_lo, double* out_hi, double* out_flo, GbState* st, const GbScan& sc,
                             cudaStream_t s) {
    unsigned tiles = grid_for(count, GB_TILE);
    if ((int)tiles > sc.max_tiles) return cudaErrorInvalidValue;
    gb_launch_count++;
    k_out_count<<<tiles, PT, 0, s>>>(E, count, gub, sc.tile_cnt, st);
    gb_launch_count++;
    k_scan_tiles<<<1, 1024, 0, s>>>(1, sc.tile_cnt, sc.tile_off, sc.max_tiles, 3, count, GbGenConst{}, st);
    gb_launch_count++;
    k_out_scatter<<<tiles, PT, 0, s>>>(E, count, gub, sc.tile_off, list);
    if (out_lo) {
        gb_launch_count++;
        k_out_gather<<<grid_for(count * 32, 128), 128, 0, s>>>(E, list, st, pool, out_lo, out_hi, out_flo);
    }
    return cudaGetLastError();
}

cudaError_t gb_launch_eval_boxes(const GbProg& P, const double* lo, const double* hi, float* scratch32,
                                 long long nbox, int blk, int fp32, double* F, double* Fmid, double* G, int* mono,
                                 cudaStream_t s) {
    float* lo32 = nullptr;
    float* hi32 = nullptr;
    if (fp32) {
        long long cnt = nbox * (long long)P.n;
        lo32 = scratch32;
        hi32 = scratch32 + cnt;
        gb_launch_count++;
        k_to_f32<<<grid_for(cnt, 256), 256, 0, s>>>(lo, hi, lo32, hi32, cnt);
    }
    gb_launch_count++;
    if (P.any_prod)
        k_eval_boxes<true><<<grid_for(nbox, 128), 128, 0, s>>>(P, lo, hi, lo32, hi32, nbox, blk, fp32, F, Fmid, G, mono);
    else
        k_eval_boxes<false><<<grid_for(nbox, 128), 128, 0, s>>>(P, lo, hi, lo32, hi32, nbox, blk, fp32, F, Fmid, G,
                                                                mono);
    return cudaGetLastError();
}

cudaError_t gb_launch_peak(int which, int iters, int blocks, void* sink, cudaStream_t s) {
    gb_launch_count++;
    if (which == 0)
        k_peak<double><<<blocks, 256, 0, s>>>(iters, 1.0, 1e-300, 1.0000001, (double*)sink);
    else
        k_peak<float><<<blocks, 256, 0, s>>>(iters, 1.0f, 1e-30f, 1.0001f, (float*)sink);
    return cudaGetLastError();
}
