// Expression-DAG -> device bytecode compiler.
//
// The objective arrives as the node array of include/gb.h.  The compiler
//  1. validates it (operator codes, topological operands, coordinate and
//     table ranges, finite constants);
//  2. splits it into the outer expression (reachable from the root without
//     entering a sum) and one template per ISUM node;
//  3. emits straight-line bytecode with one register per node, in ascending
//     node order, so that the reverse sweep (the interval gradient used by the
//     first-order test of section 3.1) walks the same list backwards;
//  4. groups the terms of every sum into maximal runs with the same range of
//     touched cycling blocks (section 3.2 cycles the split over blocks of B
//     coordinates) and records, for every block b, the run of groups whose
//     terms touch it.  A box caches one partial sum per group; a child split
//     in block b recomputes only those groups.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "gb_internal.h"

namespace {

// Outward conversion of an exact double to a float interval.
void out_float(double c, float* lo, float* hi) {
    float f = (float)c;
    *lo = ((double)f <= c) ? f : std::nextafter(f, -INFINITY);
    *hi = ((double)f >= c) ? f : std::nextafter(f, INFINITY);
}

int n_operands(int op) {
    switch (op) {
    case GB_OP_ADD: case GB_OP_SUB: case GB_OP_MUL: case GB_OP_DIV: return 2;
    case GB_OP_NEG: case GB_OP_SQR: case GB_OP_SQRT: case GB_OP_EXP: case GB_OP_SIN:
    case GB_OP_COS: case GB_OP_SCALE: case GB_OP_STEP: return 1;
    default: return 0;
    }
}

uint8_t dev_op(int op) {
    switch (op) {
    case GB_OP_CONST: return D_CONST;
    case GB_OP_PI: return D_PI;
    case GB_OP_EULER: return D_EULER;
    case GB_OP_VAR: return D_VAR;
    case GB_OP_IDX_VAR: return D_IVAR;
    case GB_OP_IDX_COEF: return D_COEF;
    case GB_OP_ADD: return D_ADD;
    case GB_OP_SUB: return D_SUB;
    case GB_OP_MUL: return D_MUL;
    case GB_OP_DIV: return D_DIV;
    case GB_OP_NEG: return D_NEG;
    case GB_OP_SQR: return D_SQR;
    case GB_OP_SQRT: return D_SQRT;
    case GB_OP_EXP: return D_EXP;
    case GB_OP_SIN: return D_SIN;
    case GB_OP_COS: return D_COS;
    case GB_OP_SCALE: return D_SCALE;
    case GB_OP_STEP: return D_STEP;
    default: return D_ISUMV;
    }
}

// Directed-rounding floating-point operations of one instruction's forward
// step (endpoint operations of the interval formula) and of its reverse step
// (the adjoint products and the accumulation into each operand).
int fwd_ops(uint8_t op) {
    switch (op) {
    case D_ADD: case D_SUB: case D_MUL: case D_SQR: case D_SCALE:
    case D_SQRT: case D_EXP: case D_SIN: case D_COS: return 2;
    case D_DIV: return 4;
    default: return 0;
    }
}
int rev_ops(uint8_t op) {
    switch (op) {
    case D_ADD: case D_SUB: return 4;               // two accumulations
    case D_MUL: return 8;                           // two products, two accumulations
    case D_DIV: return 12;
    case D_NEG: return 2;
    case D_SQR: case D_EXP: case D_SCALE: return 4; // product, accumulation
    case D_SQRT: case D_SIN: case D_COS: return 6;
    default: return 0;
    }
}

struct Ctx {
    const gb_node* nd;
    int nn;
    std::vector<char> outer, mark;
};

bool mark_outer(Ctx& c, int v, std::string& err) {
    if (c.outer[v]) return true;
    c.outer[v] = 1;
    const gb_node& q = c.nd[v];
    if (q.op == GB_OP_IDX_VAR || q.op == GB_OP_IDX_COEF) {
        err = "IDX_VAR / IDX_COEF node " + std::to_string(v) + " used outside a sum template";
        return false;
    }
    if (q.op == GB_OP_ISUM || q.op == GB_OP_IPROD) return true;
    int k = n_operands(q.op);
    if (k >= 1 && !mark_outer(c, q.a, err)) return false;
    if (k >= 2 && !mark_outer(c, q.b, err)) return false;
    return true;
}

bool mark_template(Ctx& c, int v, std::string& err) {
    if (c.mark[v]) return true;
    c.mark[v] = 1;
    const gb_node& q = c.nd[v];
    if (q.op == GB_OP_VAR || q.op == GB_OP_ISUM || q.op == GB_OP_IPROD) {
        err = "VAR / ISUM / IPROD node " + std::to_string(v) + " inside a sum template";
        return false;
    }
    int k = n_operands(q.op);
    if (k >= 1 && !mark_template(c, q.a, err)) return false;
    if (k >= 2 && !mark_template(c, q.b, err)) return false;
    return true;
}

}  // namespace

std::string gb_compile(const gb_node* nd, int32_t nn, int32_t root, const int64_t* tlen,
                       int32_t ntab, int32_t n, int32_t B, GbHostProg* P) {
    if (nn < 1 || root < 0 || root >= nn) return "root outside the node array";
    if (n < 1) return "dimension n must be >= 1";
    if (B < 1 || B > n) return "block size must satisfy 1 <= B <= n";
    if (ntab < 0) return "negative table count";
    for (int v = 0; v < nn; v++) {
        const gb_node& q = nd[v];
        if (q.op < 0 || q.op > GB_OP_STEP) return "unknown operator at node " + std::to_string(v);
        if (q.pad != 0) return "nonzero pad at node " + std::to_string(v);
        int k = n_operands(q.op);
        if (k >= 1 && (q.a < 0 || q.a >= v)) return "operand not before node " + std::to_string(v);
        if (k >= 2 && (q.b < 0 || q.b >= v)) return "operand not before node " + std::to_string(v);
        if ((q.op == GB_OP_CONST || q.op == GB_OP_SCALE) && !std::isfinite(q.v))
            return "non-finite constant at node " + std::to_string(v);
        if (q.op == GB_OP_VAR && (q.a < 0 || q.a >= n)) return "VAR coordinate out of range";
        if ((q.op == GB_OP_ISUM || q.op == GB_OP_IPROD) && (q.a < 0 || q.a >= v || q.d < 1))
            return "bad ISUM / IPROD at node " + std::to_string(v);
    }
    Ctx c{nd, nn, std::vector<char>(nn, 0), std::vector<char>(nn, 0)};
    std::string err;
    if (!mark_outer(c, root, err)) return err;

    P->n = n;
    P->B = B;
    P->nb = (n + B - 1) / B;
    P->any_prod = 0;
    P->outer.clear(); P->tins.clear(); P->sums.clear(); P->groups.clear();
    P->dirty.clear(); P->var_leaves.clear();

    std::vector<int> oreg(nn, -1);
    for (int v = 0; v < nn; v++)
        if (c.outer[v]) oreg[v] = (int)(P->outer.size()), P->outer.push_back(GbIns{});
    if ((int)P->outer.size() > GB_MAX_OREGS) return "outer expression exceeds the register limit";
    P->outer_root = oreg[root];

    for (int v = 0; v < nn; v++) {
        if (!c.outer[v]) continue;
        const gb_node& q = nd[v];
        GbIns& I = P->outer[oreg[v]];
        I = GbIns{};
        I.op = dev_op(q.op);
        I.dst = (uint8_t)oreg[v];
        int k = n_operands(q.op);
        if (k >= 1) I.a = (uint8_t)oreg[q.a];
        if (k >= 2) I.b = (uint8_t)oreg[q.b];
        I.c = q.v;
        out_float(q.v, &I.clo32, &I.chi32);
        I.pad = fwd_ops(I.op) | (rev_ops(I.op) << 8);
        if (q.op == GB_OP_VAR) {
            I.aux = q.a;
            P->var_leaves.push_back(GbVarLeaf{oreg[v], q.a});
        }
        if (q.op != GB_OP_ISUM && q.op != GB_OP_IPROD) continue;

        // ---- an ISUM / IPROD node: its template ---------------------------
        int ks = (int)P->sums.size();
        if (ks >= GB_MAX_ISUM) return "too many sums";
        I.aux = ks;
        std::fill(c.mark.begin(), c.mark.end(), 0);
        if (!mark_template(c, q.a, err)) return err;
        std::vector<int> treg(nn, -1);
        GbSum S{};
        S.prod = q.op == GB_OP_IPROD ? 1 : 0;
        if (S.prod) P->any_prod = 1;
        S.ins0 = (int)P->tins.size();
        int omin = 0, omax = 0, hv = 0, nleaf = 0;
        for (int t = 0; t <= q.a; t++) {
            if (!c.mark[t]) continue;
            treg[t] = (int)P->tins.size() - S.ins0;
            const gb_node& w = nd[t];
            GbIns J{};
            J.op = dev_op(w.op);
            J.dst = (uint8_t)treg[t];
            int kk = n_operands(w.op);
            if (kk >= 1) J.a = (uint8_t)treg[w.a];
            if (kk >= 2) J.b = (uint8_t)treg[w.b];
            J.c = w.v;
            out_float(w.v, &J.clo32, &J.chi32);
            J.pad = fwd_ops(J.op) | (rev_ops(J.op) << 8);
            if (w.op == GB_OP_IDX_VAR) {
                J.aux = w.b;
                if (!hv) omin = omax = w.b, hv = 1;
                omin = std::min(omin, w.b);
                omax = std::max(omax, w.b);
                nleaf++;
            }
            if (w.op == GB_OP_IDX_COEF) {
                if (w.a < 0 || w.a >= ntab) return "IDX_COEF table out of range";
                J.aux = w.a;
                J.aux2 = w.b;
            }
            P->tins.push_back(J);
        }
        S.nins = (int)P->tins.size() - S.ins0;
        if (S.nins > GB_MAX_TREGS) return "sum template exceeds the register limit";
        if (treg[q.a] != S.nins - 1) return "internal: template root is not last";
        S.first = q.b;
        S.step = q.d;
        S.count = q.c > q.b ? (q.c - q.b + q.d - 1) / q.d : 0;
        if (S.count >= (1 << 20)) return "sum with 2^20 or more terms";  // reduction tree depth limit
        S.off_min = omin;
        S.off_max = omax;
        S.has_var = hv;
        S.nvar_leaves = nleaf;
        S.outer_reg = oreg[v];
        if (hv && omax - omin + 1 > GB_MAX_WIN) return "IDX_VAR offsets span too wide";
        if (S.count > 0) {
            int64_t i0 = S.first, i1 = (int64_t)S.first + (int64_t)(S.count - 1) * S.step;
            if (hv && (i0 + omin < 0 || i1 + omax >= n)) return "IDX_VAR index out of range";
            for (int t = S.ins0; t < S.ins0 + S.nins; t++) {
                const GbIns& J = P->tins[t];
                if (J.op != D_COEF) continue;
                if (i0 + J.aux2 < 0 || i1 + J.aux2 >= tlen[J.aux]) return "IDX_COEF index out of range";
            }
        }
        // groups: runs of terms with the same touched-block range
        S.group0 = (int)P->groups.size();
        for (int t = 0; t < S.count; t++) {
            int i = S.first + t * S.step;
            int b0 = hv ? (i + omin) / B : -1, b1 = hv ? (i + omax) / B : -1;
            if (t == 0 || P->groups.back().bmin != b0 || P->groups.back().bmax != b1)
                P->groups.push_back(GbGroup{t, 0, b0, b1});
            P->groups.back().count++;
        }
        S.ngroups = (int)P->groups.size() - S.group0;
        P->sums.push_back(S);
    }
    // dirty group ranges per block (local indices within each sum)
    int ns = (int)P->sums.size();
    P->dirty.assign((size_t)P->nb * ns, int2{0, 0});
    for (int b = 0; b < P->nb; b++)
        for (int k = 0; k < ns; k++) {
            const GbSum& S = P->sums[k];
            int g0 = -1, g1 = -1;
            for (int g = 0; g < S.ngroups; g++) {
                const GbGroup& G = P->groups[S.group0 + g];
                if (G.bmin <= b && b <= G.bmax) {
                    if (g0 < 0) g0 = g;
                    g1 = g + 1;
                }
            }
            if (g0 < 0) g0 = g1 = 0;
            P->dirty[(size_t)b * ns + k] = int2{g0, g1};
        }

    // group ownership for the block-record pool
    {
        const int NG = (int)P->groups.size();
        P->gown.assign(NG, int2{0, 0});
        std::vector<int> cnt(P->nb, 0);
        P->span = 0;
        for (int g = 0; g < NG; g++) {
            const GbGroup& G = P->groups[g];
            const int ob = G.bmin < 0 ? 0 : G.bmin;
            if (G.bmin >= 0) P->span = std::max(P->span, G.bmax - G.bmin);
            P->gown[g] = int2{ob, cnt[ob]++};
        }
        P->GPB = 1;
        for (int b = 0; b < P->nb; b++) P->GPB = std::max(P->GPB, cnt[b]);
        P->owned.assign((size_t)P->nb * P->GPB, -1);
        for (int g = 0; g < NG; g++) P->owned[(size_t)P->gown[g].x * P->GPB + P->gown[g].y] = g;
    }

    // static directed-op counts, averaged over the blocks
    int64_t tot_eval = 0, tot_mid = 0;
    int64_t outer_f = 0, outer_r = 0;
    for (auto& I : P->outer) outer_f += fwd_ops(I.op), outer_r += rev_ops(I.op);
    for (int b = 0; b < P->nb; b++) {
        int64_t ev = outer_f + outer_r, md = outer_f;
        int c0 = b * B, c1 = std::min(n, c0 + B);
        for (int k = 0; k < ns; k++) {
            const GbSum& S = P->sums[k];
            int64_t tf = 0, tr = 0;
            for (int t = S.ins0; t < S.ins0 + S.nins; t++)
                tf += fwd_ops(P->tins[t].op), tr += rev_ops(P->tins[t].op);
            int2 dr = P->dirty[(size_t)b * ns + k];
            int64_t dterms = 0;
            for (int g = dr.x; g < dr.y; g++) dterms += P->groups[S.group0 + g].count;
            int64_t tree = 2 * std::max(0, S.ngroups - 1) + 2 * std::max<int64_t>(0, dterms - (dr.y - dr.x));
            ev += dterms * tf + tree;
            md += dterms * tf + tree + 2 * dterms * S.nvar_leaves;  // midpoint of each loaded coordinate
            if (!S.has_var) continue;
            int64_t gterms = 0;
            for (int t = 0; t < S.count; t++) {
                int i = S.first + t * S.step;
                if (i + S.off_max >= c0 && i + S.off_min < c1) gterms++;
            }
            ev += gterms * (tf + tr) + 2 * gterms * S.nvar_leaves + 2 * (c1 - c0);
        }
        tot_eval += ev;
        tot_mid += md;
    }
    P->ops_eval = tot_eval / P->nb;
    P->ops_mid = tot_mid / P->nb;
    return "";
}

// Per-split-position layouts of the per-parent term tables (see GbSplitPos).
void gb_build_tables(GbHostProg* P, int m, int d, int sbits) {
    P->tab_ok = 0;
    P->m = m;
    P->mshift = m == 2 ? 1 : 2;
    P->sp_of_cyc.assign(P->n, -1);
    P->sps.clear();
    P->dterms.clear();
    P->jk.clear();
    P->contribs.clear();
    P->jkd.clear();
    P->max_drows = 0;
    P->segs.clear();
    P->max_srows = 0;
    P->max_nseg = 0;
    P->max_rows = P->max_dterm = 0;
    if (P->any_prod) return;   // the tables hold sums only: products run on the interpreter
    const int n = P->n, B = P->B, ns = (int)P->sums.size();
    int node = 0, max_leaves = 0;
    for (GbSum& S : P->sums) {
        S.node0 = node;
        int cnt = 0;
        for (int mL = S.ngroups; mL > 0; mL = (mL + 1) / 2) {
            cnt += mL;
            if (mL == 1) break;
        }
        S.nnodes = cnt;
        node += cnt;
        max_leaves = std::max(max_leaves, S.nvar_leaves);
    }
    P->tree_nodes = node;
    P->max_leaves = max_leaves;
    for (int b = 0; b < P->nb; b++) {
        const int bs = b * B, be = std::min(n, bs + B);
        for (int c = bs; c < be; c += d) {
            const int dd = std::min(d, be - c);
            GbSplitPos sp{};
            sp.c0 = c;
            sp.dd = dd;
            sp.block = b;
            sp.dterm0 = (int)P->dterms.size();
            sp.jk0 = (int)P->jk.size();
            int rows = 0;
            for (int k = 0; k < ns; k++) {
                const GbSum& S = P->sums[k];
                int2 dr = P->dirty[(size_t)b * ns + k];
                if (dr.y - dr.x > GB_TAB_MAX_DIRTY) return;
                for (int g = dr.x; g < dr.y; g++) {
                    const GbGroup& G = P->groups[S.group0 + g];
                    for (int t = G.t0; t < G.t0 + G.count; t++) {
                        const int i = S.first + t * S.step;
                        int w = 0, a = 0;
                        if (S.has_var) {
                            a = std::max(i + S.off_min, c);
                            const int z = std::min(i + S.off_max, c + dd - 1);
                            w = a <= z ? z - a + 1 : 0;
                        }
                        GbDTerm D{};
                        D.sum = (int16_t)k;
                        D.w = (int16_t)w;
                        D.dshift = (int16_t)(w ? (a - c) * P->mshift : 0);
                        D.group = (int16_t)g;
                        D.term = t;
                        D.row = rows;
                        rows += 1 << (w * P->mshift);
                        P->dterms.push_back(D);
                    }
                }
            }
            sp.ndterm = (int)P->dterms.size() - sp.dterm0;
            sp.tab_entries = rows;
            // segments of each dirty group's term tree: greedily the largest
            // aligned block of 2^L terms whose digit bits fit GB_TAB_SBITS
            sp.seg0 = (int)P->segs.size();
            for (int q0 = 0; q0 < sp.ndterm;) {
                const GbDTerm& D0 = P->dterms[sp.dterm0 + q0];
                int cnt = 0;
                while (q0 + cnt < sp.ndterm && P->dterms[sp.dterm0 + q0 + cnt].sum == D0.sum &&
                       P->dterms[sp.dterm0 + q0 + cnt].group == D0.group)
                    cnt++;
                auto bits_of = [&](int t0, int len, int* lo_out) {
                    int lo = 1 << 30, hi = 0;
                    for (int t = t0; t < t0 + len; t++) {
                        const GbDTerm& D = P->dterms[sp.dterm0 + q0 + t];
                        if (D.w == 0) continue;
                        lo = std::min(lo, (int)D.dshift);
                        hi = std::max(hi, (int)D.dshift + D.w * P->mshift);
                    }
                    if (lo > hi) lo = hi = 0;
                    *lo_out = lo;
                    return hi - lo;
                };
                for (int t = 0; t < cnt;) {
                    int L = 0, lo = 0;
                    while (t % (2 << L) == 0 && t + (2 << L) <= cnt) {
                        const int b = bits_of(t, 2 << L, &lo);
                        if (b > sbits || b + L + 1 > GB_TAB_SCOST) break;
                        L++;
                    }
                    const GbDTerm& D = P->dterms[sp.dterm0 + q0 + t];
                    GbSeg g{};
                    g.dterm = q0 + t;
                    g.sum = (int8_t)D.sum;
                    g.group = D.group;
                    g.level = (int8_t)L;
                    if (L == 0) {
                        g.base = D.row;
                        g.shift = D.dshift;
                        g.mask = (uint16_t)((1u << (D.w * P->mshift)) - 1u);
                    } else {
                        const int b = bits_of(t, 1 << L, &lo);
                        g.base = sp.srows;
                        g.shift = (int16_t)lo;
                        g.mask = (uint16_t)((1u << b) - 1u);
                        sp.srows += 1 << b;
                    }
                    P->segs.push_back(g);
                    t += 1 << L;
                }
                q0 += cnt;
            }
            sp.nseg = (int)P->segs.size() - sp.seg0;
            P->max_srows = std::max(P->max_srows, sp.srows);
            P->max_nseg = std::max(P->max_nseg, sp.nseg);
            if (rows > GB_TAB_MAX_ROWS) return;
            P->max_rows = std::max(P->max_rows, rows);
            P->max_dterm = std::max(P->max_dterm, sp.ndterm);
            // gradient contributions of every block coordinate, per sum, in
            // ascending term and ascending leaf order
            for (int j = bs; j < be; j++) {
                for (int k = 0; k < ns; k++) {
                    const GbSum& S = P->sums[k];
                    const int start = (int)P->contribs.size();
                    if (S.has_var) {
                        for (int q = 0; q < sp.ndterm; q++) {
                            const GbDTerm& D = P->dterms[sp.dterm0 + q];
                            if (D.sum != k) continue;
                            const int i = S.first + D.term * S.step;
                            int leaf = 0;
                            for (int t = S.ins0; t < S.ins0 + S.nins; t++) {
                                if (P->tins[t].op != D_IVAR) continue;
                                if (i + P->tins[t].aux == j)
                                    P->contribs.push_back(GbContrib{q, leaf, D.row * max_leaves + leaf, D.dshift,
                                                                    (uint16_t)((1u << (D.w * P->mshift)) - 1u)});
                                leaf++;
                            }
                        }
                    }
                    const int end = (int)P->contribs.size();
                    P->jk.push_back(int2{start, end});
                    // digit bits the contributions depend on
                    GbJkD J{0, -1, 0};
                    if (end > start) {
                        int lo = 1 << 30, hi = 0;
                        for (int q = start; q < end; q++) {
                            const GbContrib& C = P->contribs[q];
                            const int nb = __builtin_popcount((unsigned)C.mask);
                            if (nb == 0) continue;
                            lo = std::min(lo, (int)C.dshift);
                            hi = std::max(hi, (int)C.dshift + nb);
                        }
                        if (lo > hi) lo = hi = 0;   // no contribution touches a split coordinate
                        if (hi - lo <= GB_TAB_DBITS) {
                            J.base = sp.drows;
                            J.shift = (int16_t)lo;
                            J.mask = (uint16_t)((1u << (hi - lo)) - 1u);
                            sp.drows += 1 << (hi - lo);
                        }
                    }
                    P->jkd.push_back(J);
                }
            }
            P->max_drows = std::max(P->max_drows, sp.drows);
            P->sp_of_cyc[c] = (int)P->sps.size();
            P->sps.push_back(sp);
        }
    }
    P->tab_ok = 1;
}
