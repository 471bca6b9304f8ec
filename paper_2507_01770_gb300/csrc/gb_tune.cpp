// Autotuner of the batching layer: the bisection fan-out (m pieces of d
// coordinates), the parents per generation and the child-kernel shape are
// chosen by timing complete solves of a representative problem.  Every
// candidate runs the same rigorous method; only the time differs.
#include <chrono>
#include <cstring>
#include <vector>

#include "gb_launch.h"

namespace {

struct Candidate {
    int m, d, parents, eval_mode;
};

std::vector<Candidate> candidates(int B) {
    std::vector<Candidate> out;
    const int halves[2] = {B, (B + 1) / 2};
    for (int m : {2, 4}) {
        const int bits = m == 2 ? 1 : 2;
        for (int hi = 0; hi < 2; hi++) {
            const int d = halves[hi];
            if (d < 1 || d * bits > GB_MAX_FAN_LOG2 || (hi == 1 && halves[1] == halves[0])) continue;
            for (int parents : {1, 4})
                for (int em : {3, 4}) out.push_back(Candidate{m, d, parents, em});
        }
    }
    return out;
}

}  // namespace

extern "C" gb_status gb_autotune(const gb_node* dag, int32_t n_nodes, int32_t root, const double* const* tables,
                                 const int64_t* table_lens, int32_t n_tables, int32_t n, const double* l,
                                 const double* u, double tol, const gb_options* base, double budget_ms,
                                 gb_options* best, double* best_ms) {
    if (!best || !best_ms || n < 1) return gb_internal_fail(GB_E_INVALID, "bad gb_autotune arguments");
    gb_options b0;
    gb_default_options(&b0);
    if (base) b0 = *base;
    const int B = b0.block > 0 ? (b0.block < n ? b0.block : n) : (n < 10 ? n : 10);
    const auto t0 = std::chrono::steady_clock::now();
    auto elapsed = [&] { return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count(); };
    bool found = false;
    gb_status last = GB_E_LIMIT;
    for (const Candidate& c : candidates(B)) {
        if (found && elapsed() >= budget_ms) break;
        gb_options o = b0;
        o.block = B;
        o.split_m = c.m;
        o.split_d = c.d;
        long long fan = 1LL << (c.d * (c.m == 2 ? 1 : 2));
        o.max_children = c.parents * fan;
        o.eval_mode = c.eval_mode;
        gb_problem* p = nullptr;
        gb_status st = gb_create_problem(dag, n_nodes, root, tables, table_lens, n_tables, n, l, u, tol, &o, &p);
        if (st != GB_OK) {
            last = st;
            continue;
        }
        double ms = 0.0;
        for (int rep = 0; rep < 2 && st == GB_OK; rep++) {   // the first solve warms up (graphs, allocator)
            gb_result r;
            std::memset(&r, 0, sizeof(r));
            st = gb_solve_device(p, &r);
            ms = r.solve_ms;
            gb_free_result(&r);
        }
        gb_destroy_problem(p);
        if (st != GB_OK) {
            last = st;
            continue;
        }
        if (!found || ms < *best_ms) {
            *best = o;
            *best_ms = ms;
            found = true;
        }
    }
    if (!found) return gb_internal_fail(last == GB_OK ? GB_E_LIMIT : last, "no autotuner candidate completed");
    return GB_OK;
}
