// C ABI of the library (include/gb.h): problem creation, the generation loop
// of the batched best-first branch and bound, result handling and the
// per-box evaluation hook.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "gb_internal.h"
#include "gb_launch.h"

namespace {

thread_local std::string g_err;

gb_status fail(gb_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

gb_status cuda_fail(cudaError_t e, const char* where) {
    g_err = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? GB_E_OOM : GB_E_CUDA;
}

#define GB_CU(call)                                        \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

// Device allocations of a problem are stream-ordered (cudaMallocAsync on the
// problem's stream, freed with cudaFreeAsync): creating and destroying
// problems never synchronises the whole device, which matters when a server
// creates and retires problems while others run.
struct DevAlloc {
    std::vector<void*>* owned;
    size_t* bytes;
    cudaStream_t s;
};

template <typename T>
cudaError_t upload(T** dst, const T* src, size_t count, DevAlloc& a) {
    *dst = nullptr;
    size_t bytes = sizeof(T) * (count ? count : 1);
    cudaError_t e = cudaMallocAsync((void**)dst, bytes, a.s);
    if (e != cudaSuccess) return e;
    a.owned->push_back(*dst);
    *a.bytes += bytes;
    if (count) e = cudaMemcpyAsync(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice, a.s);
    return e;
}

template <typename T>
cudaError_t alloc(T** dst, size_t count, DevAlloc& a) {
    *dst = nullptr;
    size_t bytes = sizeof(T) * (count ? count : 1);
    cudaError_t e = cudaMallocAsync((void**)dst, bytes, a.s);
    if (e == cudaSuccess) {
        a.owned->push_back(*dst);
        *a.bytes += bytes;
    }
    return e;
}

void float_bounds(double c, float* lo, float* hi) {
    float f = (float)c;
    *lo = ((double)f <= c) ? f : std::nextafter(f, -INFINITY);
    *hi = ((double)f >= c) ? f : std::nextafter(f, INFINITY);
}

}  // namespace

struct SolveRun {
    bool active = false, loop_done = false;
    int cur = 0;
    std::vector<gb_gen_stat> trace;
    long long last_par = 0, launches = 0;
    bool timed64 = false, timed32 = false;
    double t64 = 0.0, t32 = 0.0;
    long long n64 = 0, n32 = 0;
    gb_status status = GB_OK;
    std::chrono::steady_clock::time_point t0;
};

struct gb_problem {
    int n = 0, device = 0;
    gb_options opt{};
    double tol_f = 0.0;
    GbHostProg hp;
    GbProg P{};
    std::vector<void*> owned;      // device allocations
    cudaStream_t stream = nullptr;
    GbFork fork{};                 // second stream and events for the single parent's tables
    GbPool pool{};
    GbEntries E[2]{};
    GbParents par{};
    GbChildren ch{};
    GbScan sc{};
    GbSplit sp{};
    GbTabs tabs{};
    bool use_tabs = false;
    GbState* st = nullptr;         // device
    GbState* st_host = nullptr;    // pinned host
    unsigned* out_list = nullptr;
    long long cap = 0, K = 0, Cmax = 0, fan = 0;
    cudaEvent_t ev[6] = {};        // solve start/end, eval64 start/end, eval32 start/end
    cudaEvent_t ev_state = nullptr; // the state record of the last generation has reached the host
    SolveRun run;
    GbGenConst G{};
    gb_gen_stat* trace_dev = nullptr;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};   // gens_per_sync generations starting on pool buffer 0 / 1
    cudaGraphExec_t gpart[2][2] = {};  // fused serving: [pool buffer][before / after the child evaluation]
    long long part_kernels[2][2] = {};
    long long graph_kernels = 0;
    size_t device_bytes = 0;       // device memory held by the problem
    bool marks_used = false;       // a solve stamped record marks (cleared before the next one)
    bool have_pool = false;        // a solve has left a pool to snapshot
    std::vector<double> lo_host, hi_host;   // the bounds l, u (snapshot checks)
    long long gen_base = 0;        // generations before this solve (resumed solves)
};

extern "C" {

void gb_default_options(gb_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->split_m = 2;
    o->max_generations = 1000000000LL;
    o->max_children = 1LL << 22;
    o->pool_bytes = (size_t)16 << 30;
}

const char* gb_status_str(gb_status s) {
    switch (s) {
    case GB_OK: return "ok";
    case GB_E_INVALID: return "invalid argument";
    case GB_E_OOM: return "out of memory";
    case GB_E_CAPACITY: return "box pool capacity reached";
    case GB_E_LIMIT: return "generation limit reached";
    case GB_E_TIMEOUT: return "device wait timed out";
    case GB_E_CUDA: return "CUDA error";
    case GB_E_BUSY: return "busy";
    }
    return "unknown status";
}

const char* gb_last_error(void) { return g_err.c_str(); }

void gb_destroy_problem(gb_problem* p) {
    if (!p) return;
    cudaSetDevice(p->device);
    if (p->stream) {
        for (void* q : p->owned) cudaFreeAsync(q, p->stream);
        cudaStreamSynchronize(p->stream);
    } else {
        for (void* q : p->owned) cudaFree(q);
    }
    if (p->st_host) cudaFreeHost(p->st_host);
    for (cudaEvent_t e : p->ev)
        if (e) cudaEventDestroy(e);
    if (p->ev_state) cudaEventDestroy(p->ev_state);
    for (cudaGraphExec_t g : p->gexec)
        if (g) cudaGraphExecDestroy(g);
    for (auto& pp : p->gpart)
        for (cudaGraphExec_t g : pp)
            if (g) cudaGraphExecDestroy(g);
    if (p->fork.fork) cudaEventDestroy(p->fork.fork);
    if (p->fork.join) cudaEventDestroy(p->fork.join);
    if (p->fork.s2) cudaStreamDestroy(p->fork.s2);
    if (p->stream) cudaStreamDestroy(p->stream);
    delete p;
}

gb_status gb_create_problem(const gb_node* dag, int32_t n_nodes, int32_t root, const double* const* tables,
                            const int64_t* table_lens, int32_t n_tables, int32_t n, const double* l,
                            const double* u, double tol, const gb_options* opt_in, gb_problem** out) {
    if (!out) return fail(GB_E_INVALID, "out is NULL");
    *out = nullptr;
    if (!dag || n_nodes < 1 || n < 1 || !l || !u || n_tables < 0 || (n_tables > 0 && (!tables || !table_lens)))
        return fail(GB_E_INVALID, "missing DAG, bounds or tables");
    gb_options opt;
    gb_default_options(&opt);
    if (opt_in) opt = *opt_in;
    if (opt.split_m == 0) opt.split_m = 2;
    if (opt.max_generations <= 0) opt.max_generations = 1000000000LL;
    if (opt.max_children <= 0) opt.max_children = 1LL << 22;
    if (opt.pool_bytes == 0) opt.pool_bytes = (size_t)16 << 30;
    if (opt.block <= 0) opt.block = n < 10 ? n : 10;
    if (opt.block > n) return fail(GB_E_INVALID, "block size larger than n");
    if (opt.pool_mode < 0 || opt.pool_mode > 2) return fail(GB_E_INVALID, "pool_mode must be 0, 1 or 2");
    if (opt.eval_mode < 0 || opt.eval_mode > 4) return fail(GB_E_INVALID, "eval_mode must be 0 .. 4");
    if (opt.samples < 0 || opt.samples > 64) return fail(GB_E_INVALID, "samples must be 0 .. 64");
    if (opt.samples > 0 || opt.mono_all) {   // paper mode: full evaluations in the interpreter
        if (opt.eval_mode >= 2) return fail(GB_E_INVALID, "samples > 0 and mono_all need eval_mode 0 or 1");
        opt.eval_mode = 1;
    }
    if (opt.max_records < 0) return fail(GB_E_INVALID, "max_records must be >= 0");
    if (opt.split_m != 2 && opt.split_m != 4) return fail(GB_E_INVALID, "split_m must be 2 or 4");
    const int mshift = opt.split_m == 2 ? 1 : 2;
    if (opt.split_d <= 0) {
        opt.split_d = opt.block;
        while (opt.split_d > 1 && (opt.split_d * mshift > 12 || opt.split_d > GB_MAX_SPLIT_D)) opt.split_d--;
    }
    if (opt.split_d > opt.block || opt.split_d > GB_MAX_SPLIT_D || opt.split_d * mshift > GB_MAX_FAN_LOG2)
        return fail(GB_E_INVALID, "split_d must be <= block, <= 20 and give at most 2^20 children per parent");
    double tol_f = opt.tol_f > 0.0 ? opt.tol_f : tol;
    if (!(tol_f >= 0.0) || !std::isfinite(tol_f)) return fail(GB_E_INVALID, "tolerance must be finite and >= 0");
    if (!(opt.tol_x >= 0.0)) return fail(GB_E_INVALID, "tol_x must be >= 0");
    for (int j = 0; j < n; j++)
        if (!std::isfinite(l[j]) || !std::isfinite(u[j]) || !(l[j] < u[j]) || !std::isfinite(u[j] - l[j]))
            return fail(GB_E_INVALID, "bounds must be finite with l < u (coordinate " + std::to_string(j) + ")");
    for (int t = 0; t < n_tables; t++) {
        if (table_lens[t] < 0 || (table_lens[t] > 0 && !tables[t])) return fail(GB_E_INVALID, "bad table");
        for (int64_t i = 0; i < table_lens[t]; i++)
            if (!std::isfinite(tables[t][i])) return fail(GB_E_INVALID, "non-finite coefficient");
    }

    gb_problem* p = new gb_problem();
    p->n = n;
    p->lo_host.assign(l, l + n);
    p->hi_host.assign(u, u + n);
    p->opt = opt;
    p->tol_f = tol_f;
    p->device = opt.device;
    std::string err = gb_compile(dag, n_nodes, root, table_lens, n_tables, n, opt.block, &p->hp);
    if (!err.empty()) {
        delete p;
        return fail(GB_E_INVALID, err);
    }
    if (p->hp.any_prod) {   // products run on the bytecode interpreter only
        if (opt.eval_mode >= 2) {
            delete p;
            return fail(GB_E_INVALID, "IPROD problems need eval_mode 0 or 1");
        }
        p->opt.eval_mode = opt.eval_mode = 1;
    }
    // term-table layouts also set each sum's tree offsets: build them before
    // the program is uploaded
    if (opt.eval_mode != 1) {
        // segment tables are per parent: the widest segments whose tables for
        // all parents of a generation fit max(64 MiB, pool budget / 8)
        const int msh = opt.split_m == 2 ? 1 : 2;
        const long long fan = 1LL << (opt.split_d * msh);
        const long long K = std::max(1LL, (long long)opt.max_children / fan);
        const double budget = std::max(64.0 * (1 << 20), (double)opt.pool_bytes / 8.0);
        const double per_row = opt.fp32_prefilter ? 40.0 : 32.0;
        for (int sbits = GB_TAB_SBITS; sbits >= 0; sbits--) {
            gb_build_tables(&p->hp, opt.split_m, opt.split_d, sbits);
            if (!p->hp.tab_ok || (double)K * p->hp.max_srows * per_row <= budget) break;
        }
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= opt.device || opt.device < 0) {
        delete p;
        return fail(GB_E_CUDA, "no CUDA device available");
    }
    cudaError_t e = cudaSetDevice(opt.device);
    if (e != cudaSuccess) {
        delete p;
        return cuda_fail(e, "cudaSetDevice");
    }
    gb_status rc = GB_OK;
    auto bad = [&](cudaError_t ee, const char* where) {
        rc = cuda_fail(ee, where);
        gb_destroy_problem(p);
        return rc;
    };
    if ((e = cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking))) return bad(e, "cudaStreamCreate");
    if ((e = cudaStreamCreateWithFlags(&p->fork.s2, cudaStreamNonBlocking)) ||
        (e = cudaEventCreateWithFlags(&p->fork.fork, cudaEventDisableTiming)) ||
        (e = cudaEventCreateWithFlags(&p->fork.join, cudaEventDisableTiming)))
        return bad(e, "cudaStreamCreate");
    DevAlloc A{&p->owned, &p->device_bytes, p->stream};

    // ---- program and tables ----------------------------------------------
    const GbHostProg& H = p->hp;
    GbProg& P = p->P;
    P.n = n;
    P.B = H.B;
    P.nb = H.nb;
    P.n_sum = (int)H.sums.size();
    P.n_groups = (int)H.groups.size();
    P.n_outer = (int)H.outer.size();
    P.outer_root = H.outer_root;
    P.n_var_leaves = (int)H.var_leaves.size();
    P.outer_sum = (H.outer.size() == 1 && H.outer[0].op == D_ISUMV && H.outer_root == 0 && !H.any_prod) ? 1 : 0;
    {
        // the outer adjoints that are exact constants: the root's is [1, 1];
        // an addition passes its adjoint to both operands, a subtraction to
        // the left one (the right one gets its negation), a negation its
        // negation; anything else makes its operands' adjoints data-dependent
        const int no = (int)H.outer.size();
        std::vector<double> adj(no, 0.0);
        std::vector<char> known(no, 1);
        if (no > 0) adj[H.outer_root] = 1.0;
        auto pass = [&](int r, double v, bool k) {
            if (r < 0 || r >= no) return;
            if (!k) known[r] = 0;
            else adj[r] += v;
        };
        for (int t = no - 1; t >= 0; t--) {
            const GbIns& I = H.outer[t];
            const bool k = known[t] != 0;
            switch (I.op) {
            case D_ADD: pass(I.a, adj[t], k); pass(I.b, adj[t], k); break;
            case D_SUB: pass(I.a, adj[t], k); pass(I.b, -adj[t], k); break;
            case D_NEG: pass(I.a, -adj[t], k); break;
            case D_CONST: case D_PI: case D_EULER: case D_VAR: case D_ISUMV: break;
            default: pass(I.a, 0.0, false); pass(I.b, 0.0, false); break;
            }
        }
        bool unit = !H.any_prod && H.var_leaves.empty() && !H.sums.empty();
        for (const GbSum& S : H.sums) unit = unit && known[S.outer_reg] && adj[S.outer_reg] == 1.0;
        P.outer_unit = unit ? 1 : 0;
    }
    P.any_prod = H.any_prod;
    P.samples = opt.samples;
    P.mono_all = opt.mono_all ? 1 : 0;
    GbIns *d_outer, *d_tins;
    GbSum* d_sums;
    GbGroup* d_groups;
    int2* d_dirty;
    GbVarLeaf* d_leaves;
    double *d_l, *d_u;
    if ((e = upload(&d_outer, H.outer.data(), H.outer.size(), A))) return bad(e, "upload program");
    if ((e = upload(&d_tins, H.tins.data(), H.tins.size(), A))) return bad(e, "upload program");
    if ((e = upload(&d_sums, H.sums.data(), H.sums.size(), A))) return bad(e, "upload program");
    if ((e = upload(&d_groups, H.groups.data(), H.groups.size(), A))) return bad(e, "upload program");
    if ((e = upload(&d_dirty, H.dirty.data(), H.dirty.size(), A))) return bad(e, "upload program");
    if ((e = upload(&d_leaves, H.var_leaves.data(), H.var_leaves.size(), A))) return bad(e, "upload program");
    if ((e = upload(&d_l, l, (size_t)n, A))) return bad(e, "upload bounds");
    if ((e = upload(&d_u, u, (size_t)n, A))) return bad(e, "upload bounds");
    std::vector<const double*> t64(n_tables > 0 ? n_tables : 1, nullptr);  // kept until the final sync
    std::vector<const float2*> t32(n_tables > 0 ? n_tables : 1, nullptr);
    for (int t = 0; t < n_tables; t++) {
        double* d64;
        float2* d32;
        std::vector<float2> f(table_lens[t]);
        for (int64_t i = 0; i < table_lens[t]; i++) float_bounds(tables[t][i], &f[i].x, &f[i].y);
        if ((e = upload(&d64, tables[t], (size_t)table_lens[t], A))) return bad(e, "upload tables");
        if ((e = upload(&d32, f.data(), f.size(), A))) return bad(e, "upload tables");
        if ((e = cudaStreamSynchronize(p->stream))) return bad(e, "upload tables");   // f is released below
        t64[t] = d64;
        t32[t] = d32;
    }
    const double** d_t64;
    const float2** d_t32;
    if ((e = upload(&d_t64, t64.data(), t64.size(), A))) return bad(e, "upload tables");
    if ((e = upload(&d_t32, t32.data(), t32.size(), A))) return bad(e, "upload tables");
    P.outer = d_outer;
    P.tins = d_tins;
    P.sums = d_sums;
    P.groups = d_groups;
    P.dirty = d_dirty;
    P.var_leaves = d_leaves;
    P.tab64 = d_t64;
    P.tab32 = d_t32;
    P.l = d_l;
    P.u = d_u;
    int2* d_gown;
    int32_t* d_owned;
    if ((e = upload(&d_gown, H.gown.data(), H.gown.size(), A)) ||
        (e = upload(&d_owned, H.owned.data(), H.owned.size(), A)))
        return bad(e, "upload group ownership");
    P.GPB = H.GPB;
    P.span = H.span;
    P.nrec = std::min(H.nb, H.span + 1);
    P.gown = d_gown;
    P.owned = d_owned;

    // ---- solver buffers ------------------------------------------------------
    const int m = opt.split_m, d = opt.split_d;
    p->fan = 1LL << (d * mshift);
    p->Cmax = (opt.max_children / p->fan) * p->fan;
    if (p->Cmax < p->fan) p->Cmax = p->fan;
    p->K = p->Cmax / p->fan;
    p->sp = GbSplit{m, mshift, d, d * mshift, d};
    const int fp32 = opt.fp32_prefilter ? 1 : 0;
    const int NG = P.n_groups > 0 ? P.n_groups : 1;
    GbPool& pl = p->pool;
    pl.n = n;
    pl.NG = NG;
    pl.fp32 = fp32;
    // box storage: dense rows, or block records when n >= 128 and a child
    // replaces few of the blocks (a record holds B coordinates and the cached sums of the
    // groups its block owns; records per box budgeted at 4 * nrec)
    const int nrec = std::min(H.nb, H.span + 1);
    // paper mode caches per-box sample sums and coordinate partials in dense rows
    const bool paper = opt.samples > 0 || opt.mono_all;
    const bool recs = opt.pool_mode == 2 || (opt.pool_mode == 0 && !paper && n >= 128 && 4 * nrec <= H.nb);
    long long cap = 0;
    // widest IDX_VAR offset range of a template: 0 when every term reads one coordinate
    int tw = 0;
    for (const GbSum& S : H.sums)
        if (S.has_var) tw = std::max(tw, S.off_max - S.off_min);
    if (recs) {
        // paper mode on records: sample sums per owned group; the coordinate
        // partials of a record's block only when no template reaches across
        // coordinates (then they depend on the record's coordinates alone)
        const bool rdp = opt.mono_all && P.n_sum > 0 && !H.any_prod && tw == 0;
        const size_t per_slot = (size_t)H.nb * 4 + 4 + 4 + 2 * 16;
        const size_t per_rec = (size_t)opt.block * (16 + (fp32 ? 8 : 0)) + (size_t)H.GPB * (32 + (fp32 ? 8 : 0)) + 4 + 1 + 4 +
                               (size_t)opt.samples * H.GPB * 16 + (rdp ? (size_t)P.n_sum * opt.block * 16 : 0);
        const long long rho = 4LL * nrec;
        cap = opt.max_boxes > 0 ? opt.max_boxes : (long long)(opt.pool_bytes / (per_slot + rho * per_rec));
        if (cap < 1) return bad(cudaErrorMemoryAllocation, "pool budget below one box");
        if (cap > (1LL << 31) - 1) cap = (1LL << 31) - 1;
        long long R = opt.max_records > 0 ? opt.max_records : cap * rho + H.nb;
        if (R > (1LL << 32) - 64) R = (1LL << 32) - 64;
        if (R < H.nb) return bad(cudaErrorMemoryAllocation, "record capacity below the root box's blocks");
        pl.recs = 1;
        pl.nb = H.nb;
        pl.B = opt.block;
        pl.GPB = H.GPB;
        pl.nrec = nrec;
        pl.R = R;
        const size_t RB = (size_t)R * opt.block, RG = (size_t)R * H.GPB;
        if ((e = alloc(&pl.rid, (size_t)cap * H.nb, A)) || (e = alloc(&pl.swide, (size_t)cap, A)) ||
            (e = alloc(&pl.freel, (size_t)cap, A)) || (e = alloc(&pl.rlo, RB, A)) || (e = alloc(&pl.rhi, RB, A)) ||
            (e = alloc(&pl.rgsum, RG, A)) || (e = alloc(&pl.rgmid, RG, A)) || (e = alloc(&pl.rfree, (size_t)R, A)) ||
            (e = alloc(&pl.rwide, (size_t)R, A)) || (e = alloc(&pl.rmark, (size_t)R, A)))
            return bad(e, "allocate block records");
        if (fp32 && ((e = alloc(&pl.rlo32, RB, A)) || (e = alloc(&pl.rhi32, RB, A)) ||
                     (e = alloc(&pl.rgsum32, RG, A))))
            return bad(e, "allocate block records");
        if (opt.samples > 0) {
            pl.S = opt.samples;
            if ((e = alloc(&pl.rgsamp, RG * (size_t)opt.samples, A))) return bad(e, "allocate block records");
        }
        if (rdp && (e = alloc(&pl.rgdp, (size_t)R * P.n_sum * opt.block, A))) return bad(e, "allocate block records");
        if ((e = cudaMemsetAsync(pl.rmark, 0, sizeof(unsigned) * (size_t)R, p->stream)))
            return bad(e, "cudaMemset");
    } else {
        size_t per_slot = (size_t)n * 16 + (fp32 ? (size_t)n * 8 : 0) + (size_t)NG * 32 + (fp32 ? (size_t)NG * 8 : 0) +
                          4 + 2 * 16 + (size_t)opt.samples * NG * 16 +
                          (opt.mono_all && !H.any_prod ? (size_t)P.n_sum * n * 16 : 0);
        cap = opt.max_boxes > 0 ? opt.max_boxes : (long long)(opt.pool_bytes / per_slot);
        if (cap < 1) return bad(cudaErrorMemoryAllocation, "pool budget below one box");
        if (cap > (1LL << 31) - 1) cap = (1LL << 31) - 1;
        if ((e = alloc(&pl.lo64, (size_t)cap * n, A)) || (e = alloc(&pl.hi64, (size_t)cap * n, A)) ||
            (e = alloc(&pl.gsum, (size_t)cap * NG, A)) || (e = alloc(&pl.gmid, (size_t)cap * NG, A)) ||
            (e = alloc(&pl.freel, (size_t)cap, A)))
            return bad(e, "allocate box pool");
        if (fp32) {
            if ((e = alloc(&pl.lo32, (size_t)cap * n, A)) || (e = alloc(&pl.hi32, (size_t)cap * n, A)) ||
                (e = alloc(&pl.gsum32, (size_t)cap * NG, A)))
                return bad(e, "allocate box pool");
        }
        if (opt.mono_all && P.n_sum > 0 && !H.any_prod) {   // cached coordinate partials (sums only)
            if ((e = alloc(&pl.gdp, (size_t)cap * P.n_sum * n, A))) return bad(e, "allocate box pool");
        }
        if (opt.samples > 0) {   // cached group sums at every diagonal sample
            pl.S = opt.samples;
            if ((e = alloc(&pl.gsamp, (size_t)cap * opt.samples * NG, A))) return bad(e, "allocate box pool");
        }
    }
    p->cap = cap;
    for (int b = 0; b < 2; b++)
        if ((e = alloc(&p->E[b].flo, (size_t)cap, A)) || (e = alloc(&p->E[b].slot, (size_t)cap, A)) ||
            (e = alloc(&p->E[b].cyc, (size_t)cap, A)))
            return bad(e, "allocate pool entries");
    const size_t K = (size_t)p->K, bt = K * d * (m + 1);
    if ((e = alloc(&p->par.slot, K, A)) || (e = alloc(&p->par.cyc, K, A)) ||
        (e = alloc(&p->par.flo, K, A)) || (e = alloc(&p->par.info, K, A)) ||
        (e = alloc(&p->par.bnd, bt, A)) || (e = alloc(&p->par.bnd_rd, bt, A)) ||
        (e = alloc(&p->par.bnd_ru, bt, A)))
        return bad(e, "allocate parent buffers");
    const size_t C = (size_t)p->Cmax;
    if ((e = alloc(&p->ch.flo, C, A)) || (e = alloc(&p->ch.flag, C, A)) ||
        (e = alloc(&p->ch.flag32, C, A)) || (e = alloc(&p->ch.list32, C, A)) ||
        (e = alloc(&p->ch.surv, C, A)))
        return bad(e, "allocate child buffers");
    // per-parent term tables
    if (opt.eval_mode != 1) {
        const bool want = opt.eval_mode >= 2 || p->fan >= 16;
        if (p->hp.tab_ok && want) {
            const GbHostProg& Hh = p->hp;
            int32_t* d_spc;
            GbSplitPos* d_sps;
            GbDTerm* d_dt;
            int2* d_jk;
            GbContrib* d_cb;
            GbJkD* d_jkd;
            GbSeg* d_segs;
            if ((e = upload(&d_jkd, Hh.jkd.data(), Hh.jkd.size(), A)) ||
                (e = upload(&d_segs, Hh.segs.data(), Hh.segs.size(), A)) ||
                (e = upload(&d_spc, Hh.sp_of_cyc.data(), Hh.sp_of_cyc.size(), A)) ||
                (e = upload(&d_sps, Hh.sps.data(), Hh.sps.size(), A)) ||
                (e = upload(&d_dt, Hh.dterms.data(), Hh.dterms.size(), A)) ||
                (e = upload(&d_jk, Hh.jk.data(), Hh.jk.size(), A)) ||
                (e = upload(&d_cb, Hh.contribs.data(), Hh.contribs.size(), A)))
                return bad(e, "upload table layouts");
            P.tab_ok = 1;
            P.m = Hh.m;
            P.mshift = Hh.mshift;
            P.max_rows = Hh.max_rows;
            P.max_leaves = Hh.max_leaves > 0 ? Hh.max_leaves : 1;
            P.tree_nodes = Hh.tree_nodes > 0 ? Hh.tree_nodes : 1;
            P.max_dterm = Hh.max_dterm;
            P.sp_of_cyc = d_spc;
            P.sps = d_sps;
            P.dterms = d_dt;
            P.jk = d_jk;
            P.contribs = d_cb;
            P.jkd = d_jkd;
            P.max_drows = Hh.max_drows > 0 ? Hh.max_drows : 1;
            P.segs = d_segs;
            P.max_srows = Hh.max_srows > 0 ? Hh.max_srows : 1;
            P.max_nseg = Hh.max_nseg;
            GbTabs& T = p->tabs;
            T.max_rows = P.max_rows > 0 ? P.max_rows : 1;
            T.max_leaves = P.max_leaves;
            T.tree_nodes = P.tree_nodes;
            T.max_drows = P.max_drows;
            T.max_srows = P.max_srows;
            if ((e = alloc(&T.ts64, K * (size_t)T.max_srows, A)) || (e = alloc(&T.tsm64, K * (size_t)T.max_srows, A)) ||
                (fp32 && (e = alloc(&T.ts32, K * (size_t)T.max_srows, A))))
                return bad(e, "allocate segment tables");
            const size_t rows = K * (size_t)T.max_rows, nodes = K * (size_t)T.tree_nodes;
            if ((e = alloc(&T.td64, K * (size_t)T.max_drows, A)) ||
                (fp32 && (e = alloc(&T.td32, K * (size_t)T.max_drows, A))))
                return bad(e, "allocate partial tables");
            if ((e = alloc(&T.tv64, rows, A)) || (e = alloc(&T.tm64, rows, A)) ||
                (e = alloc(&T.tl64, rows * T.max_leaves, A)) || (e = alloc(&T.nf64, nodes, A)) ||
                (e = alloc(&T.nm64, nodes, A)))
                return bad(e, "allocate term tables");
            if (fp32 && ((e = alloc(&T.tv32, rows, A)) || (e = alloc(&T.tl32, rows * T.max_leaves, A)) ||
                         (e = alloc(&T.nf32, nodes, A))))
                return bad(e, "allocate term tables");
            T.warp = opt.eval_mode == 4 ? 1 : opt.eval_mode == 3 ? 0 : (gb_warp_per_child(p->Cmax) ? 1 : 0);
            T.reg = 0;
            if (P.outer_sum && P.n_sum == 1 && P.n_var_leaves == 0) {   // the register-resident walk of the one sum
                const GbSum& S0 = Hh.sums[0];
                bool fits = true;
                for (int b = 0; b < Hh.nb && fits; b++) {
                    const int2 dr = Hh.dirty[b];
                    fits = dr.y - dr.x <= GB_REG_DIRTY;
                    for (int g = dr.x; g < dr.y && fits; g++)
                        fits = Hh.groups[S0.group0 + g].count < (1 << GB_REG_LEVELS);
                }
                T.reg = fits ? 1 : 0;
            }
            T.max_sum_nodes = 1;
            for (const GbSum& S : Hh.sums) T.max_sum_nodes = std::max(T.max_sum_nodes, (int)S.nnodes);
            // no opt-in needed: the table kernel's static shared memory (about 7 KB) and the
            // trees stay within the 48 KB a launch gets by default
            T.tree_smem = (size_t)T.max_sum_nodes * sizeof(double2) <= 32 * 1024 ? 1 : 0;
            if (T.warp) {   // per-child sums and dirty group values (k_child_sums)
                const size_t cs = (size_t)p->Cmax * (P.n_sum > 0 ? P.n_sum : 1), cg = (size_t)p->Cmax * GB_CG;
                if ((e = alloc(&T.cs64, cs, A)) || (e = alloc(&T.csm64, cs, A)) || (e = alloc(&T.cg64, cg, A)) ||
                    (e = alloc(&T.cgm64, cg, A)) || (fp32 && ((e = alloc(&T.cs32, cs, A)) || (e = alloc(&T.cg32, cg, A)))))
                    return bad(e, "allocate child sums");
                if ((P.outer_unit || (P.outer_sum && P.n_sum == 1)) && P.n_var_leaves == 0) {   // verdict tables
                    const size_t mv = (size_t)p->K * P.B << GB_MV_BITS;
                    if ((e = alloc(&T.mv64, mv, A)) || (fp32 && (e = alloc(&T.mv32, mv, A))) ||
                        (e = alloc(&T.mvb, (size_t)p->K * P.B, A)))
                        return bad(e, "allocate first-order verdicts");
                }
            }
            p->use_tabs = true;
        }
    }
    p->G.K = p->K;
    p->G.flog2 = d * mshift;
    p->G.fp32 = fp32;
    p->G.max_gen = opt.max_generations;
    p->G.tol_f = tol_f;
    p->G.tol_x = opt.tol_x;
    p->G.trace_cap = opt.max_generations < (1LL << 20) ? opt.max_generations : (1LL << 20);
    p->G.nrec = pl.recs ? pl.nrec : 0;
    p->G.R = pl.recs ? pl.R : 0;
    if ((e = alloc(&p->trace_dev, (size_t)p->G.trace_cap, A))) return bad(e, "allocate trace");
    p->G.trace = p->trace_dev;
    long long items = std::max(std::max(cap, p->Cmax), pl.recs ? pl.R : 0LL);
    p->sc.max_tiles = (int)((items + GB_TILE - 1) / GB_TILE) + 1;
    if ((e = alloc(&p->sc.tile_cnt, (size_t)3 * p->sc.max_tiles, A)) ||
        (e = alloc(&p->sc.tile_off, (size_t)3 * p->sc.max_tiles, A)) ||
        (e = alloc(&p->sc.hist, (size_t)65536, A)) || (e = alloc(&p->out_list, (size_t)cap, A)) ||
        (e = alloc(&p->sc.tile_flag, (size_t)p->sc.max_tiles, A)) ||
        (e = alloc(&p->sc.stat_key, (size_t)GB_STAT_BLOCKS, A)) ||
        (e = alloc(&p->sc.stat_pos, (size_t)GB_STAT_BLOCKS, A)) ||
        (e = alloc(&p->st, 1, A)))
        return bad(e, "allocate scan buffers");
    if ((e = cudaMemsetAsync(p->sc.hist, 0, 65536 * sizeof(unsigned), p->stream))) return bad(e, "cudaMemset");
    if ((e = cudaMallocHost((void**)&p->st_host, sizeof(GbState)))) return bad(e, "cudaMallocHost");
    for (cudaEvent_t& ev : p->ev)
        if ((e = cudaEventCreate(&ev))) return bad(e, "cudaEventCreate");
    if ((e = cudaEventCreateWithFlags(&p->ev_state, cudaEventDisableTiming))) return bad(e, "cudaEventCreate");
    if ((e = cudaStreamSynchronize(p->stream))) return bad(e, "upload");   // host sources may now go away
    *out = p;
    return GB_OK;
}

gb_status gb_problem_info(const gb_problem* p, int32_t* block, int32_t* n_blocks, int64_t* ops_eval,
                          int64_t* ops_mid) {
    if (!p) return fail(GB_E_INVALID, "NULL problem");
    if (block) *block = p->hp.B;
    if (n_blocks) *n_blocks = p->hp.nb;
    if (ops_eval) *ops_eval = p->hp.ops_eval;
    if (ops_mid) *ops_mid = p->hp.ops_mid;
    return GB_OK;
}

void gb_free_result(gb_result* r) {
    if (!r) return;
    std::free(r->box_lo);
    std::free(r->box_hi);
    std::free(r->box_flo);
    std::free(r->trace);
    std::memset(r, 0, sizeof(*r));
}

// ---------------------------------------------------------------------------
// A solve as a resumable state machine: solve_begin enqueues the root box,
// each solve_advance reads the state record of the previous generation (when
// its asynchronous copy has landed) and enqueues the next generation,
// solve_finish gathers the output.  gb_solve runs the three blocking; the
// serving loop interleaves many problems without blocking on any of them.
static gb_status solve_begin_from(gb_problem* p, const gb_snapshot* snap) {
    SolveRun& R = p->run;
    R = SolveRun{};
    R.t0 = std::chrono::steady_clock::now();
    GB_CU(cudaSetDevice(p->device));
    const long long l0 = gb_launches_so_far();
    cudaStream_t s = p->stream;
    GbState init{};
    init.cap = p->cap;
    GB_CU(cudaEventRecord(p->ev[0], s));
    GB_CU(cudaMemcpyAsync(p->st, &init, sizeof(GbState), cudaMemcpyHostToDevice, s));
    // the pool partitions' tile flags carry an epoch that restarts with every solve
    GB_CU(cudaMemsetAsync(p->sc.tile_flag, 0, sizeof(unsigned long long) * (size_t)p->sc.max_tiles, s));
    if (p->pool.recs && p->marks_used) {   // collection numbers restart at 1 in every solve
        GB_CU(cudaMemsetAsync(p->pool.rmark, 0, sizeof(unsigned) * (size_t)p->pool.R, s));
        p->marks_used = false;
    }
    p->have_pool = false;
    if (!snap) {
        p->gen_base = 0;
        GB_CU(gb_launch_root_init(p->P, p->pool, p->E[0], p->G.tol_x, p->st, s));
    } else {   // regions of a snapshot: upload, enter the pool, recompute their caches
        p->gen_base = snap->generations;
        const long long c = snap->count;
        const size_t nb = (size_t)c * p->n;
        double *d_lo = nullptr, *d_hi = nullptr, *d_flo = nullptr;
        int* d_cyc = nullptr;
        cudaError_t e = cudaSuccess;
        if (c > 0) {
            cudaError_t e1 = cudaMallocAsync((void**)&d_lo, nb * sizeof(double), s);
            cudaError_t e2 = cudaMallocAsync((void**)&d_hi, nb * sizeof(double), s);
            cudaError_t e3 = cudaMallocAsync((void**)&d_flo, (size_t)c * sizeof(double), s);
            cudaError_t e4 = cudaMallocAsync((void**)&d_cyc, (size_t)c * sizeof(int), s);
            e = e1 ? e1 : e2 ? e2 : e3 ? e3 : e4;
            if (e == cudaSuccess &&
                (e = cudaMemcpyAsync(d_lo, snap->lo, nb * sizeof(double), cudaMemcpyHostToDevice, s)) == cudaSuccess &&
                (e = cudaMemcpyAsync(d_hi, snap->hi, nb * sizeof(double), cudaMemcpyHostToDevice, s)) == cudaSuccess &&
                (e = cudaMemcpyAsync(d_flo, snap->flo, (size_t)c * sizeof(double), cudaMemcpyHostToDevice, s)) ==
                    cudaSuccess)
                e = cudaMemcpyAsync(d_cyc, snap->cyc, (size_t)c * sizeof(int), cudaMemcpyHostToDevice, s);
        }
        if (e == cudaSuccess)
            e = gb_launch_resume(p->P, p->pool, p->E[0], c, d_lo, d_hi, d_flo, d_cyc, snap->gub, p->st, s);
        if (d_lo) cudaFreeAsync(d_lo, s);
        if (d_hi) cudaFreeAsync(d_hi, s);
        if (d_flo) cudaFreeAsync(d_flo, s);
        if (d_cyc) cudaFreeAsync(d_cyc, s);
        if (e != cudaSuccess) return cuda_fail(e, "resume from a snapshot");
    }
    GB_CU(gb_launch_stats(p->E[0], p->G, 1, p->sc, p->st, s));
    GB_CU(cudaMemcpyAsync(p->st_host, p->st, sizeof(GbState), cudaMemcpyDeviceToHost, s));
    GB_CU(cudaEventRecord(p->ev_state, s));
    R.launches += gb_launches_so_far() - l0;
    R.active = true;
    p->have_pool = true;
    return GB_OK;
}

__attribute__((visibility("hidden"))) gb_status solve_begin(gb_problem* p) { return solve_begin_from(p, nullptr); }

// Captures gens_per_sync consecutive generations as one CUDA graph per
// starting pool buffer (once per problem; every argument of a generation is
// fixed, sizes come from the device state, and a generation that must not
// run is skipped by all its kernels), so the host launches one graph per
// state read.
static cudaError_t capture_graphs(gb_problem* p) {
    cudaStream_t s = p->stream;
    const int G = p->opt.gens_per_sync;
    for (int par = 0; par < 2; par++) {
        if (p->gexec[par]) continue;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        long long nl = 0;
        for (int k = 0; k < G && e == cudaSuccess; k++) {
            const int b = (par + k) & 1;
            long long n1 = 0;
            e = gb_launch_generation(p->P, p->pool, p->E[b], p->E[1 - b], p->par, p->ch, p->sp, p->sc,
                                     p->use_tabs ? &p->tabs : nullptr, p->G, p->cap, p->Cmax, p->st, s, nullptr,
                                     &n1, 0, &p->fork);
            nl += n1;
        }
        cudaError_t e2 = cudaStreamEndCapture(s, &g);
        if (e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return e;
        }
        if (e2 != cudaSuccess) return e2;
        e = cudaGraphInstantiate(&p->gexec[par], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return e;
        p->graph_kernels = nl;
    }
    return cudaSuccess;
}

// Returns 1 when the generation loop has ended (R.status holds the outcome),
// 0 when more generations were enqueued or (non-blocking) the previous ones
// have not finished yet.
// 1: the loop has ended (R.status holds the outcome); 0: the previous
// generation has finished and the next may be enqueued; -1: it has not
// finished yet (non-blocking).  Reading the same state again gives the same
// answer.
__attribute__((visibility("hidden"))) int solve_check(gb_problem* p, bool block) {
    SolveRun& R = p->run;
    if (R.loop_done) return 1;
    auto stop = [&](gb_status st) {
        R.status = st;
        R.loop_done = true;
        return 1;
    };
    cudaError_t q = block ? cudaEventSynchronize(p->ev_state) : cudaEventQuery(p->ev_state);
    if (q == cudaErrorNotReady) return -1;
    if (q != cudaSuccess) return stop(cuda_fail(q, "generation"));
    cudaSetDevice(p->device);
    const GbState h = *p->st_host;
    float ms = 0.f;
    if (R.timed64 && cudaEventElapsedTime(&ms, p->ev[2], p->ev[3]) == cudaSuccess) R.t64 += ms, R.n64++;
    if (R.timed32 && cudaEventElapsedTime(&ms, p->ev[4], p->ev[5]) == cudaSuccess) R.t32 += ms, R.n32++;
    R.timed64 = R.timed32 = false;
    if (h.error) return stop(fail(GB_E_CUDA, "device-side selection error"));
    if (h.overflow)
        return stop(fail(GB_E_CAPACITY, p->pool.recs ? "box pool or block record capacity reached"
                                                      : "box pool capacity reached"));
    if (h.active == 0) return stop(GB_OK);
    if (h.halt || h.gen >= p->opt.max_generations) return stop(fail(GB_E_LIMIT, "generation limit reached"));
    return 0;
}

__attribute__((visibility("hidden"))) int solve_advance(gb_problem* p, bool block) {
    SolveRun& R = p->run;
    const int c = solve_check(p, block);
    if (c != 0) return c > 0 ? 1 : 0;
    auto stop = [&](gb_status st) {
        R.status = st;
        R.loop_done = true;
        return 1;
    };
    cudaStream_t s = p->stream;
    const GbState h = *p->st_host;
    const long long l0 = gb_launches_so_far();
    const int cur = (int)(h.gen & 1);   // every completed generation swaps the pool buffers
    cudaError_t e = cudaSuccess;
    const int G = p->opt.gens_per_sync;
    if (G > 1) {
        if ((e = capture_graphs(p)) != cudaSuccess) return stop(cuda_fail(e, "graph capture"));
        if ((e = cudaGraphLaunch(p->gexec[cur], s)) != cudaSuccess) return stop(cuda_fail(e, "cudaGraphLaunch"));
        R.launches += p->graph_kernels;
    } else {
        long long nl = 0;
        e = gb_launch_generation(p->P, p->pool, p->E[cur], p->E[1 - cur], p->par, p->ch, p->sp, p->sc,
                                 p->use_tabs ? &p->tabs : nullptr, p->G, p->cap, p->Cmax, p->st, s, &p->ev[2], &nl, 0,
                                 &p->fork);
        if (e != cudaSuccess) return stop(cuda_fail(e, "generation launch"));
        R.timed64 = true;
        R.timed32 = p->opt.fp32_prefilter != 0;
        R.launches += gb_launches_so_far() - l0;
    }
    if ((e = cudaMemcpyAsync(p->st_host, p->st, sizeof(GbState), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return stop(cuda_fail(e, "state readback"));
    if ((e = cudaEventRecord(p->ev_state, s)) != cudaSuccess) return stop(cuda_fail(e, "event"));
    return 0;
}

__attribute__((visibility("hidden"))) gb_status solve_finish(gb_problem* p, gb_result* out, bool copy_boxes) {
    SolveRun& R = p->run;
    std::memset(out, 0, sizeof(*out));
    GB_CU(cudaSetDevice(p->device));
    const long long l0 = gb_launches_so_far();
    cudaStream_t s = p->stream;
    GB_CU(cudaStreamSynchronize(s));
    GbState h = *p->st_host;
    const int cur = (int)(h.gen & 1);
    double gub = gb_key_value(h.gub_key);
    unsigned long long ones = ~0ull;
    GB_CU(cudaMemcpyAsync(&p->st->glb_key, &ones, sizeof(ones), cudaMemcpyHostToDevice, s));
    GB_CU(gb_launch_output(p->E[cur], h.pool, p->pool, gub, p->out_list, nullptr, nullptr, nullptr, p->st, p->sc, s));
    GB_CU(cudaMemcpyAsync(p->st_host, p->st, sizeof(GbState), cudaMemcpyDeviceToHost, s));
    GB_CU(cudaStreamSynchronize(s));
    GbState hf = *p->st_host;
    const long long nbox = hf.kept;
    out->n = p->n;
    out->n_boxes = nbox;
    out->fmin_hi = gub;
    out->fmin_lo = hf.glb_key == ~0ull ? -INFINITY : gb_key_value(hf.glb_key);
    out->generations = hf.gen;
    out->box_evals_fp32 = hf.evals32;
    out->box_evals_fp64 = hf.evals64;
    out->mid_evals = hf.mids;
    out->eval64_ms = R.t64;
    out->eval32_ms = R.t32;
    out->eval64_launches = R.n64;
    out->eval32_launches = R.n32;
    if (copy_boxes && nbox > 0) {
        size_t nb = (size_t)nbox * p->n;
        double *d_lo = nullptr, *d_hi = nullptr, *d_flo = nullptr;
        cudaError_t e1 = cudaMallocAsync((void**)&d_lo, nb * sizeof(double), s);
        cudaError_t e2 = cudaMallocAsync((void**)&d_hi, nb * sizeof(double), s);
        cudaError_t e3 = cudaMallocAsync((void**)&d_flo, (size_t)nbox * sizeof(double), s);
        if (e1 || e2 || e3) return cuda_fail(e1 ? e1 : (e2 ? e2 : e3), "allocate output");
        GB_CU(gb_launch_output(p->E[cur], h.pool, p->pool, gub, p->out_list, d_lo, d_hi, d_flo, p->st, p->sc, s));
        out->box_lo = (double*)std::malloc(nb * sizeof(double));
        out->box_hi = (double*)std::malloc(nb * sizeof(double));
        out->box_flo = (double*)std::malloc((size_t)nbox * sizeof(double));
        if (!out->box_lo || !out->box_hi || !out->box_flo) return fail(GB_E_OOM, "host allocation");
        GB_CU(cudaMemcpyAsync(out->box_lo, d_lo, nb * sizeof(double), cudaMemcpyDeviceToHost, s));
        GB_CU(cudaMemcpyAsync(out->box_hi, d_hi, nb * sizeof(double), cudaMemcpyDeviceToHost, s));
        GB_CU(cudaMemcpyAsync(out->box_flo, d_flo, (size_t)nbox * sizeof(double), cudaMemcpyDeviceToHost, s));
        cudaFreeAsync(d_lo, s);
        cudaFreeAsync(d_hi, s);
        cudaFreeAsync(d_flo, s);
        GB_CU(cudaStreamSynchronize(s));
    }
    GB_CU(cudaEventRecord(p->ev[1], s));
    GB_CU(cudaEventSynchronize(p->ev[1]));
    {
        float ms = 0.f;
        GB_CU(cudaEventElapsedTime(&ms, p->ev[0], p->ev[1]));
        out->device_ms = ms;
    }
    R.launches += gb_launches_so_far() - l0;
    out->kernel_launches = R.launches;
    out->ops64 = (int64_t)hf.ops64;
    out->ops32 = (int64_t)hf.ops32;
    out->pool_mode = p->pool.recs ? 2 : 1;
    out->record_gcs = (int64_t)hf.rec_gc;
    if (hf.rec_gc > 0) p->marks_used = true;
    const long long nt = hf.gen < p->G.trace_cap ? hf.gen : p->G.trace_cap;
    out->n_trace = nt;
    if (nt > 0) {
        out->trace = (gb_gen_stat*)std::malloc((size_t)nt * sizeof(gb_gen_stat));
        if (!out->trace) return fail(GB_E_OOM, "host allocation");
        GB_CU(cudaMemcpy(out->trace, p->trace_dev, (size_t)nt * sizeof(gb_gen_stat), cudaMemcpyDeviceToHost));
    }
    out->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - R.t0).count();
    out->status = R.status;
    R.active = false;
    return R.status;
}

// ---------------------------------------------------------------------------
// Fused evaluation over several problems (serving): a step runs G
// generations of every problem it holds together -- per generation, each
// problem's selection, partition and term tables on its own stream, then one
// persistent launch evaluating the children of all of them, then each
// problem's compaction, materialisation and statistics on its own stream.
#define GB_BATCH_RING 8   // descriptor buffers in flight (steps overlap)
struct GbBatchCtx {
    cudaStream_t ss[GB_BATCH_RING] = {};   // step i launches on ss[i % ring]: steps overlap
    cudaEvent_t ev_ev[GB_BATCH_RING] = {};
    std::vector<cudaEvent_t> ev_pre;
    GbEvalDesc* h = nullptr;   // pinned [GB_BATCH_RING][GB_BATCH_MAX]
    GbEvalDesc* d = nullptr;   // device, same shape
    cudaEvent_t ev_slot[GB_BATCH_RING] = {};   // the fused launch that last read each buffer
    int next = 0;
};

__attribute__((visibility("hidden"))) GbBatchCtx* batch_create(int device) {
    if (cudaSetDevice(device) != cudaSuccess) return nullptr;
    GbBatchCtx* B = new GbBatchCtx();
    bool ok = true;
    for (int i = 0; ok && i < GB_BATCH_RING; i++)
        ok = cudaStreamCreateWithFlags(&B->ss[i], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&B->ev_ev[i], cudaEventDisableTiming) == cudaSuccess;
    ok = ok &&
              cudaMallocHost((void**)&B->h, sizeof(GbEvalDesc) * GB_BATCH_MAX * GB_BATCH_RING) == cudaSuccess &&
              cudaMalloc((void**)&B->d, sizeof(GbEvalDesc) * GB_BATCH_MAX * GB_BATCH_RING) == cudaSuccess;
    B->ev_pre.assign(GB_BATCH_MAX, nullptr);
    for (int i = 0; ok && i < GB_BATCH_MAX; i++)
        ok = cudaEventCreateWithFlags(&B->ev_pre[i], cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; ok && i < GB_BATCH_RING; i++)
        ok = cudaEventCreateWithFlags(&B->ev_slot[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        batch_destroy(B);
        return nullptr;
    }
    return B;
}

__attribute__((visibility("hidden"))) void batch_destroy(GbBatchCtx* B) {
    if (!B) return;
    for (cudaStream_t s : B->ss)
        if (s) cudaStreamSynchronize(s);
    for (cudaEvent_t e : B->ev_pre)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : B->ev_ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : B->ev_slot)
        if (e) cudaEventDestroy(e);
    if (B->h) cudaFreeHost(B->h);
    if (B->d) cudaFree(B->d);
    for (cudaStream_t s : B->ss)
        if (s) cudaStreamDestroy(s);
    delete B;
}

__attribute__((visibility("hidden"))) void solve_abort(gb_problem* p, gb_status st) {
    p->run.status = st;
    p->run.loop_done = true;
}

// Problems whose child evaluation is the FP32-then-FP64 warp-per-child table
// kernel can join a fused launch.
__attribute__((visibility("hidden"))) bool solve_fusable(const gb_problem* p) {
    return p->use_tabs && p->tabs.warp && p->G.fp32 && p->opt.fp32_prefilter;
}

// The part (1: before, 2: after the child evaluation) of a generation that
// starts on pool buffer cur, captured once per problem as a CUDA graph
// (every size comes from the device state) and launched on its stream.
static cudaError_t launch_part(gb_problem* p, int cur, int part, long long* nl) {
    cudaGraphExec_t& gx = p->gpart[cur][part - 1];
    if (!gx) {
        cudaStream_t s = p->stream;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        long long n1 = 0;
        e = gb_launch_generation(p->P, p->pool, p->E[cur], p->E[1 - cur], p->par, p->ch, p->sp, p->sc, &p->tabs,
                                 p->G, p->cap, p->Cmax, p->st, s, nullptr, &n1, part, &p->fork);
        cudaError_t e2 = cudaStreamEndCapture(s, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&gx, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) return e;
        p->part_kernels[cur][part - 1] = n1;
    }
    *nl = p->part_kernels[cur][part - 1];
    return cudaGraphLaunch(gx, p->stream);
}

// G consecutive generations of every problem in probs (each fusable, its
// previous generation finished: solve_check returned 0), one fused
// child-evaluation launch per generation; a problem whose search ends inside
// the run skips its remaining generations (every kernel checks st->halt),
// as in a graph of G generations.  The state is read back after the last.
__attribute__((visibility("hidden"))) gb_status batch_generation(gb_problem* const* probs, int k, GbBatchCtx* B,
                                                                int G) {
    if (k <= 0) return GB_OK;
    if (k > GB_BATCH_MAX) return fail(GB_E_INVALID, "too many problems for one fused launch");
    if (G < 1) G = 1;
    for (int g = 0; g < G; g++) {
        // a descriptor buffer whose last fused launch has finished
        const int slot = B->next;
        B->next = (B->next + 1) % GB_BATCH_RING;
        GB_CU(cudaEventSynchronize(B->ev_slot[slot]));
        GbEvalDesc* hd = B->h + (size_t)slot * GB_BATCH_MAX;
        GbEvalDesc* dd = B->d + (size_t)slot * GB_BATCH_MAX;
        cudaStream_t bs = B->ss[slot];
        cudaEvent_t ev_eval = B->ev_ev[slot];
        long long units = 0;   // work units the step can hold (children per generation at most)
        for (int i = 0; i < k; i++) {
            gb_problem* p = probs[i];
            const int cur = (int)((p->st_host->gen + g) & 1);
            long long nl = 0;
            GB_CU(launch_part(p, cur, 1, &nl));
            GB_CU(cudaEventRecord(B->ev_pre[i], p->stream));
            hd[i] = GbEvalDesc{p->P, p->pool, p->par, p->tabs, p->ch, p->sp, p->st};
            p->run.launches += nl + 1;   // + its share of the fused launch
            units += (p->Cmax + 3) / 4;
        }
        GB_CU(cudaMemcpyAsync(dd, hd, sizeof(GbEvalDesc) * (size_t)k, cudaMemcpyHostToDevice, bs));
        for (int i = 0; i < k; i++) GB_CU(cudaStreamWaitEvent(bs, B->ev_pre[i], 0));
        GB_CU(gb_launch_eval3264_batch(dd, k, units, bs));
        GB_CU(cudaEventRecord(ev_eval, bs));
        GB_CU(cudaEventRecord(B->ev_slot[slot], bs));
        for (int i = 0; i < k; i++) {
            gb_problem* p = probs[i];
            const int cur = (int)((p->st_host->gen + g) & 1);
            long long nl = 0;
            GB_CU(cudaStreamWaitEvent(p->stream, ev_eval, 0));
            GB_CU(launch_part(p, cur, 2, &nl));
            p->run.launches += nl;
        }
    }
    for (int i = 0; i < k; i++) {
        gb_problem* p = probs[i];
        GB_CU(cudaMemcpyAsync(p->st_host, p->st, sizeof(GbState), cudaMemcpyDeviceToHost, p->stream));
        GB_CU(cudaEventRecord(p->ev_state, p->stream));
    }
    return GB_OK;
}

static gb_status solve_impl(gb_problem* p, gb_result* out, bool copy_boxes, const gb_snapshot* snap = nullptr) {
    if (!p || !out) return fail(GB_E_INVALID, "NULL argument");
    std::memset(out, 0, sizeof(*out));
    if (p->run.active) return fail(GB_E_BUSY, "a solve of this problem is in progress");
    gb_status st = solve_begin_from(p, snap);
    if (st != GB_OK) return st;
    while (!solve_advance(p, true)) {
    }
    gb_status fin = solve_finish(p, out, copy_boxes);
    return fin;
}

// The status of a solve goes into the result on every return path, so a
// caller that reads out->status sees a failure (whose result holds no
// enclosure) as well as the return code does.
static gb_status with_status(gb_result* out, gb_status rc) {
    if (out) out->status = rc;
    return rc;
}

gb_status gb_solve(gb_problem* p, gb_result* out) { return with_status(out, solve_impl(p, out, true)); }

gb_status gb_solve_device(gb_problem* p, gb_result* out) { return with_status(out, solve_impl(p, out, false)); }

gb_status gb_snapshot_take(gb_problem* p, gb_snapshot* out) {
    if (!p || !out) return fail(GB_E_INVALID, "NULL argument");
    std::memset(out, 0, sizeof(*out));
    if (p->run.active) return fail(GB_E_BUSY, "a solve of this problem is in progress");
    if (!p->have_pool) return fail(GB_E_INVALID, "no solve has run on this problem");
    GB_CU(cudaSetDevice(p->device));
    cudaStream_t s = p->stream;
    GB_CU(cudaStreamSynchronize(s));
    const GbState h = *p->st_host;   // state after the last solve's output pass (pool and gen unchanged)
    const long long c = h.pool;
    const int cur = (int)(h.gen & 1);
    out->n = p->n;
    out->block = p->hp.B;
    out->count = c;
    out->gub = gb_key_value(h.gub_key);
    out->generations = p->gen_base + h.gen;
    if (c == 0) return GB_OK;
    const size_t nb = (size_t)c * p->n;
    double *d_lo = nullptr, *d_hi = nullptr, *d_flo = nullptr;
    int* d_cyc = nullptr;
    cudaError_t e1 = cudaMallocAsync((void**)&d_lo, nb * sizeof(double), s);
    cudaError_t e2 = cudaMallocAsync((void**)&d_hi, nb * sizeof(double), s);
    cudaError_t e3 = cudaMallocAsync((void**)&d_flo, (size_t)c * sizeof(double), s);
    cudaError_t e4 = cudaMallocAsync((void**)&d_cyc, (size_t)c * sizeof(int), s);
    out->lo = (double*)std::malloc(nb * sizeof(double));
    out->hi = (double*)std::malloc(nb * sizeof(double));
    out->flo = (double*)std::malloc((size_t)c * sizeof(double));
    out->cyc = (int32_t*)std::malloc((size_t)c * sizeof(int32_t));
    gb_status rc = GB_OK;
    if (e1 || e2 || e3 || e4) rc = fail(GB_E_OOM, "device allocation for the snapshot");
    else if (!out->lo || !out->hi || !out->flo || !out->cyc) rc = fail(GB_E_OOM, "host allocation");
    cudaError_t e = cudaSuccess;
    if (rc == GB_OK) {
        if ((e = gb_launch_snapshot(p->E[cur], c, p->pool, d_lo, d_hi, d_flo, d_cyc, s)) == cudaSuccess &&
            (e = cudaMemcpyAsync(out->lo, d_lo, nb * sizeof(double), cudaMemcpyDeviceToHost, s)) == cudaSuccess &&
            (e = cudaMemcpyAsync(out->hi, d_hi, nb * sizeof(double), cudaMemcpyDeviceToHost, s)) == cudaSuccess &&
            (e = cudaMemcpyAsync(out->flo, d_flo, (size_t)c * sizeof(double), cudaMemcpyDeviceToHost, s)) ==
                cudaSuccess &&
            (e = cudaMemcpyAsync(out->cyc, d_cyc, (size_t)c * sizeof(int), cudaMemcpyDeviceToHost, s)) == cudaSuccess)
            e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(e, "snapshot");
    }
    if (d_lo) cudaFreeAsync(d_lo, s);
    if (d_hi) cudaFreeAsync(d_hi, s);
    if (d_flo) cudaFreeAsync(d_flo, s);
    if (d_cyc) cudaFreeAsync(d_cyc, s);
    if (rc != GB_OK) gb_free_snapshot(out);
    return rc;
}

static gb_status solve_resume_impl(gb_problem* p, const gb_snapshot* snap, gb_result* out) {
    if (!p || !snap || !out) return fail(GB_E_INVALID, "NULL argument");
    std::memset(out, 0, sizeof(*out));
    if (snap->n != p->n) return fail(GB_E_INVALID, "snapshot dimension differs from the problem's");
    if (snap->count < 0 || (snap->count > 0 && (!snap->lo || !snap->hi || !snap->flo || !snap->cyc)))
        return fail(GB_E_INVALID, "malformed snapshot");
    if (snap->gub != snap->gub) return fail(GB_E_INVALID, "snapshot GUB is NaN");
    if (p->pool.recs) return fail(GB_E_INVALID, "resume needs dense rows (pool_mode 1)");
    if (snap->count > p->cap) return fail(GB_E_CAPACITY, "snapshot regions exceed the pool capacity");
    const int n = p->n;
    for (long long q = 0; q < snap->count; q++) {
        const int c = snap->cyc[q] & 0x7fffffff;
        if (c < 0 || c >= n) return fail(GB_E_INVALID, "snapshot cycling word out of range");
        if (snap->flo[q] != snap->flo[q]) return fail(GB_E_INVALID, "snapshot lower bound is NaN");
        const double* lo = snap->lo + (size_t)q * n;
        const double* hi = snap->hi + (size_t)q * n;
        for (int j = 0; j < n; j++)
            if (!(lo[j] <= hi[j]) || !(lo[j] >= p->lo_host[j]) || !(hi[j] <= p->hi_host[j]))
                return fail(GB_E_INVALID, "snapshot region outside the bounds (or lo > hi) at region " +
                                              std::to_string(q));
    }
    return solve_impl(p, out, true, snap);
}

gb_status gb_solve_resume(gb_problem* p, const gb_snapshot* snap, gb_result* out) {
    return with_status(out, solve_resume_impl(p, snap, out));
}

void gb_free_snapshot(gb_snapshot* snap) {
    if (!snap) return;
    std::free(snap->lo);
    std::free(snap->hi);
    std::free(snap->flo);
    std::free(snap->cyc);
    std::memset(snap, 0, sizeof(*snap));
}

gb_status gb_eval_boxes(gb_problem* p, const double* d_lo, const double* d_hi, int64_t nbox, int32_t blk,
                        int32_t fp32, double* d_F, double* d_Fmid, double* d_G, int32_t* d_mono, void* stream) {
    if (!p) return fail(GB_E_INVALID, "NULL problem");
    if (nbox < 0 || blk >= p->hp.nb || (nbox > 0 && (!d_lo || !d_hi || !d_F || !d_Fmid)) ||
        (blk >= 0 && nbox > 0 && (!d_G || !d_mono)))
        return fail(GB_E_INVALID, "bad arguments to gb_eval_boxes");
    if (nbox == 0) return GB_OK;
    GB_CU(cudaSetDevice(p->device));
    cudaStream_t s = (cudaStream_t)stream;
    float* scratch = nullptr;
    if (fp32) {
        size_t cnt = (size_t)nbox * p->n * 2;
        GB_CU(cudaMallocAsync((void**)&scratch, cnt * sizeof(float), s));
    }
    cudaError_t e = gb_launch_eval_boxes(p->P, d_lo, d_hi, scratch, nbox, blk, fp32, d_F, d_Fmid, d_G, d_mono, s);
    if (scratch) cudaFreeAsync(scratch, s);
    if (e != cudaSuccess) return cuda_fail(e, "gb_eval_boxes launch");
    return GB_OK;
}

// Read-only view of a problem for the other translation units of the library
// (not exported from the shared object).
__attribute__((visibility("hidden"))) size_t gb_internal_device_bytes(const gb_problem* p) {
    return p ? p->device_bytes : 0;
}

__attribute__((visibility("hidden"))) const GbProg* gb_internal_prog(const gb_problem* p, int* device, int* n, int* nb) {
    if (!p) return nullptr;
    *device = p->device;
    *n = p->n;
    *nb = p->hp.nb;
    return &p->P;
}

// Sets the calling thread's gb_last_error() message (not exported).
__attribute__((visibility("hidden"))) gb_status gb_internal_fail(gb_status s, const char* msg) {
    return fail(s, msg);
}

gb_status gb_measure_peak(int32_t device, int32_t which, double* ops_per_s, double* ms_out) {
    if (!ops_per_s || (which != 0 && which != 1)) return fail(GB_E_INVALID, "bad arguments to gb_measure_peak");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return fail(GB_E_CUDA, "no CUDA device available");
    GB_CU(cudaSetDevice(device));
    int sms = 0;
    GB_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    const int blocks = sms * 8, iters = which == 0 ? 20000 : 200000;
    void* sink = nullptr;
    GB_CU(cudaMalloc(&sink, 256 * sizeof(double)));
    cudaEvent_t a, b;
    GB_CU(cudaEventCreate(&a));
    GB_CU(cudaEventCreate(&b));
    GB_CU(gb_launch_peak(which, 100, blocks, sink, 0));   // warm-up
    GB_CU(cudaEventRecord(a, 0));
    GB_CU(gb_launch_peak(which, iters, blocks, sink, 0));
    GB_CU(cudaEventRecord(b, 0));
    GB_CU(cudaEventSynchronize(b));
    float ms = 0.f;
    GB_CU(cudaEventElapsedTime(&ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    double ops = 8.0 * iters * (double)blocks * 256.0;
    *ops_per_s = ops / (ms * 1e-3);
    if (ms_out) *ms_out = ms;
    return GB_OK;
}

}  // extern "C"
