/*
 * CPU oracle for the interval branch-and-bound global minimiser.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, scalar restatement
 * of the method for checking the CUDA library; only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may build or call it.  It shares
 * no code, header or table with the CUDA path: it parses the objective's
 * node array (the input format) with its own definitions below.
 *
 * What it follows (Zhang, Shan, Cagan, "Global optimization tailored for
 * graphics processing units"):
 *   - interval +, -, x, / : Eqs. 3-6 (section 2.1), with optimal outward
 *     rounding of every endpoint (section 2.1): lower endpoints rounded toward
 *     -inf, upper toward +inf, here by switching the FPU mode with fesetround.
 *   - natural interval extension of f (section 2.1): each node of the
 *     objective replaced by its interval operation.
 *   - the iteration of section 3.1: sample (GUB update), remove suboptimal
 *     regions (LB > GUB), partition, rule out by cut-off and by the
 *     first-order (monotonicity) test, insert, stop; output GLB, GUB and the
 *     remaining regions.
 *   - uniform partition of the selected coordinates (Eqs. 10-11) and the
 *     variable-cycling schedule (section 3.2).
 * Where the paper leaves a choice open (reduction order, transcendental
 * rounding, sample point, batching of the best-first selection) the oracle
 * takes the readings written beside each function.
 *
 * Build: gcc -O1 -frounding-math -ffp-contract=off -fno-fast-math
 *        -fno-math-errno -pthread -shared -fPIC oracle.c -lm
 * No claim of speed is made; every directed operation is its own call.  The
 * per-child loops of a generation may run on several threads (each with its
 * own scratch and its own rounding mode, results in per-child slots), which
 * changes nothing in what is computed.
 */
#include <fenv.h>
#include <pthread.h>
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* GCC does not implement the FENV_ACCESS pragma; -frounding-math is its
 * equivalent and is required when building this file. */

#define NOINL __attribute__((noinline))

/* ------------------------------------------------------------------------ */
/* Directed rounding, section 2.1 ("optimal outward rounding").              */
/* Every helper switches the mode, performs one operation, and restores      */
/* round-to-nearest so that libm calls elsewhere run in their default mode.  */
/* ------------------------------------------------------------------------ */
static NOINL double d_add(double a, double b, int up) {
    fesetround(up ? FE_UPWARD : FE_DOWNWARD);
    volatile double r = a + b;
    fesetround(FE_TONEAREST);
    return r;
}
static NOINL double d_sub(double a, double b, int up) {
    fesetround(up ? FE_UPWARD : FE_DOWNWARD);
    volatile double r = a - b;
    fesetround(FE_TONEAREST);
    return r;
}
static NOINL double d_mul(double a, double b, int up) {
    fesetround(up ? FE_UPWARD : FE_DOWNWARD);
    volatile double r = a * b;
    fesetround(FE_TONEAREST);
    return r;
}
static NOINL double d_div(double a, double b, int up) {
    fesetround(up ? FE_UPWARD : FE_DOWNWARD);
    volatile double r = a / b;
    fesetround(FE_TONEAREST);
    return r;
}
static NOINL double d_sqrt(double a, int up) {
    fesetround(up ? FE_UPWARD : FE_DOWNWARD);
    volatile double r = __builtin_sqrt(a);
    fesetround(FE_TONEAREST);
    return r;
}
static NOINL float f_add(float a, float b, int up) {
    fesetround(up ? FE_UPWARD : FE_DOWNWARD);
    volatile float r = a + b;
    fesetround(FE_TONEAREST);
    return r;
}
static NOINL float f_sub(float a, float b, int up) {
    fesetround(up ? FE_UPWARD : FE_DOWNWARD);
    volatile float r = a - b;
    fesetround(FE_TONEAREST);
    return r;
}
static NOINL float f_mul(float a, float b, int up) {
    fesetround(up ? FE_UPWARD : FE_DOWNWARD);
    volatile float r = a * b;
    fesetround(FE_TONEAREST);
    return r;
}
static NOINL float f_div(float a, float b, int up) {
    fesetround(up ? FE_UPWARD : FE_DOWNWARD);
    volatile float r = a / b;
    fesetround(FE_TONEAREST);
    return r;
}
static NOINL float f_sqrt(float a, int up) {
    fesetround(up ? FE_UPWARD : FE_DOWNWARD);
    volatile float r = __builtin_sqrtf(a);
    fesetround(FE_TONEAREST);
    return r;
}
/* double -> float conversion rounded down (up = 0) or up (up = 1). */
static NOINL float f_conv(double a, int up) {
    fesetround(up ? FE_UPWARD : FE_DOWNWARD);
    volatile float r = (float)a;
    fesetround(FE_TONEAREST);
    return r;
}

/* Precision-generic wrappers.  In single precision (p = 1) every value held
 * in a double is a float value, so the (float) casts below are exact. */
static double R_add(double a, double b, int p, int up) {
    return p ? (double)f_add((float)a, (float)b, up) : d_add(a, b, up);
}
static double R_sub(double a, double b, int p, int up) {
    return p ? (double)f_sub((float)a, (float)b, up) : d_sub(a, b, up);
}
static double R_mul(double a, double b, int p, int up) {
    /* closed interval system: 0 * (+-inf) = 0 */
    if (a == 0.0 || b == 0.0) return 0.0;
    return p ? (double)f_mul((float)a, (float)b, up) : d_mul(a, b, up);
}
static double R_div(double a, double b, int p, int up) {
    return p ? (double)f_div((float)a, (float)b, up) : d_div(a, b, up);
}
static double R_sqrt(double a, int p, int up) {
    return p ? (double)f_sqrt((float)a, up) : d_sqrt(a, up);
}
/* Outward conversion of an FP64 number into the working precision. */
static double R_in(double a, int p, int up) {
    return p ? (double)f_conv(a, up) : a;
}
/* Move x by k units in the last place toward -inf (up = 0) or +inf. */
static double R_step(double x, int k, int p, int up) {
    for (int i = 0; i < k; i++) {
        if (p) x = (double)nextafterf((float)x, up ? INFINITY : -INFINITY);
        else   x = nextafter(x, up ? INFINITY : -INFINITY);
    }
    return x;
}

/* ------------------------------------------------------------------------ */
/* Intervals                                                                 */
/* ------------------------------------------------------------------------ */
typedef struct { double lo, hi; } iv;

static iv mk(double lo, double hi) { iv r = {lo, hi}; return r; }
static iv entire(void) { return mk(-INFINITY, INFINITY); }

/* Unit step H(y) = 1 for y >= 0, 0 for y < 0 (the indicator that builds the
 * discontinuous test function of SI Appendix F, Eq. S24): exact on an
 * interval wholly on one side of 0, [0, 1] on one that holds the jump. */
static iv iv_step(iv x) {
    if (x.lo >= 0.0) return mk(1.0, 1.0);
    if (x.hi < 0.0) return mk(0.0, 0.0);
    return mk(0.0, 1.0);
}

/* Whether the box of x holds the jump of H (its derivative is then not
 * bounded there). */
static int step_jump(iv x) { return !(x.lo >= 0.0) && !(x.hi < 0.0); }

/* Eq. 3 */
static iv iv_add(iv x, iv y, int p) {
    return mk(R_add(x.lo, y.lo, p, 0), R_add(x.hi, y.hi, p, 1));
}
/* Eq. 4 */
static iv iv_sub(iv x, iv y, int p) {
    return mk(R_sub(x.lo, y.hi, p, 0), R_sub(x.hi, y.lo, p, 1));
}
/* Eq. 5: min / max of the four endpoint products, each rounded outward. */
static iv iv_mul(iv x, iv y, int p) {
    double l1 = R_mul(x.lo, y.lo, p, 0), l2 = R_mul(x.lo, y.hi, p, 0);
    double l3 = R_mul(x.hi, y.lo, p, 0), l4 = R_mul(x.hi, y.hi, p, 0);
    double h1 = R_mul(x.lo, y.lo, p, 1), h2 = R_mul(x.lo, y.hi, p, 1);
    double h3 = R_mul(x.hi, y.lo, p, 1), h4 = R_mul(x.hi, y.hi, p, 1);
    return mk(fmin(fmin(l1, l2), fmin(l3, l4)), fmax(fmax(h1, h2), fmax(h3, h4)));
}
/* 1/[y] for Eq. 6.  Reading: when 0 lies in [y] the result is the whole
 * real line (rigorous; the paper does not treat this case). */
static iv iv_recip(iv y, int p) {
    if (y.lo > 0.0 || y.hi < 0.0)
        return mk(R_div(1.0, y.hi, p, 0), R_div(1.0, y.lo, p, 1));
    return entire();
}
/* Eq. 6: [x]/[y] = [x] * (1/[y]). */
static iv iv_div(iv x, iv y, int p) { return iv_mul(x, iv_recip(y, p), p); }

static iv iv_neg(iv x) { return mk(-x.hi, -x.lo); }

/* Square with the dependence of x*x removed (section 2.1 names the
 * dependence problem; the paper does not define sqr itself). */
static iv iv_sqr(iv x, int p) {
    if (x.lo >= 0.0) return mk(R_mul(x.lo, x.lo, p, 0), R_mul(x.hi, x.hi, p, 1));
    if (x.hi <= 0.0) return mk(R_mul(x.hi, x.hi, p, 0), R_mul(x.lo, x.lo, p, 1));
    return mk(0.0, fmax(R_mul(x.lo, x.lo, p, 1), R_mul(x.hi, x.hi, p, 1)));
}

/* sqrt restricted to its domain x >= 0; IEEE sqrt is correctly rounded in
 * each direction. */
static iv iv_sqrt(iv x, int p) {
    return mk(R_sqrt(fmax(x.lo, 0.0), p, 0), R_sqrt(fmax(x.hi, 0.0), p, 1));
}

/* Multiplication by a point constant c (exact FP64 in the problem data). */
static iv iv_scale(iv x, double c, int p) {
    if (p) {
        iv cc = mk(R_in(c, 1, 0), R_in(c, 1, 1));
        return iv_mul(x, cc, 1);
    }
    if (c == 0.0) return mk(0.0, 0.0);
    if (c > 0.0) return mk(R_mul(x.lo, c, 0, 0), R_mul(x.hi, c, 0, 1));
    return mk(R_mul(x.hi, c, 0, 0), R_mul(x.lo, c, 0, 1));
}

/* Transcendentals.  libm is called in round-to-nearest and the result is
 * widened by K_WIDEN units in the last place in each direction: glibc
 * documents at most 1 ulp of error for exp, sin and cos in both precisions,
 * and one more ulp is added as margin.  The paper is silent on how it rounds
 * transcendental functions (section 2.1 only defines outward rounding). */
#define K_WIDEN (2 + g_extra_widen)

/* Extra widening of every transcendental endpoint, in ulps (0 in every use
 * but one test, which perturbs the library values this way to check the
 * deviation bound further down against an actual deviation). */
static int g_extra_widen = 0;

static double PI_LO, PI_HI, E_LO, E_HI;      /* adjacent doubles around pi, e */

static void init_constants(void) {
    /* 0x400921FB54442D18 is the double nearest pi and lies below pi;
       0x4005BF0A8B145769 is the double nearest e and lies below e. */
    union { uint64_t u; double d; } v;
    v.u = 0x400921FB54442D18ull; PI_LO = v.d; PI_HI = nextafter(PI_LO, INFINITY);
    v.u = 0x4005BF0A8B145769ull; E_LO = v.d;  E_HI = nextafter(E_LO, INFINITY);
}

static iv const_pi(int p) { return mk(R_in(PI_LO, p, 0), R_in(PI_HI, p, 1)); }
static iv const_e(int p) { return mk(R_in(E_LO, p, 0), R_in(E_HI, p, 1)); }

static double lm_exp(double x, int p) { return p ? (double)expf((float)x) : exp(x); }
static double lm_cos(double x, int p) { return p ? (double)cosf((float)x) : cos(x); }
static double lm_sin(double x, int p) { return p ? (double)sinf((float)x) : sin(x); }

static iv iv_exp(iv x, int p) {
    double lo = R_step(lm_exp(x.lo, p), K_WIDEN, p, 0);
    double hi = R_step(lm_exp(x.hi, p), K_WIDEN, p, 1);
    if (lo < 0.0) lo = 0.0;
    return mk(lo, hi);
}

static int is_even(double k) { return fmod(k, 2.0) == 0.0; }

/* Interval cosine (cos_not_sin = 1) or sine.  Endpoint values widened as
 * above; an extremum +-1 is included whenever a critical point may lie in
 * [x] according to an outward enclosure of x/pi; wide or huge arguments
 * give [-1, 1]. */
static iv iv_trig(iv x, int p, int cos_not_sin) {
    double big = p ? 1048576.0 : 1099511627776.0; /* 2^20 / 2^40 */
    iv pi = const_pi(p);
    double w = R_sub(x.hi, x.lo, p, 1);
    double two_pi_lo = pi.lo * 2.0;
    if (!(w < two_pi_lo) || !(fabs(x.lo) <= big) || !(fabs(x.hi) <= big))
        return mk(-1.0, 1.0);
    double va = cos_not_sin ? lm_cos(x.lo, p) : lm_sin(x.lo, p);
    double vb = cos_not_sin ? lm_cos(x.hi, p) : lm_sin(x.hi, p);
    double lo = fmin(R_step(va, K_WIDEN, p, 0), R_step(vb, K_WIDEN, p, 0));
    double hi = fmax(R_step(va, K_WIDEN, p, 1), R_step(vb, K_WIDEN, p, 1));
    /* enclosure [qlo, qhi] of {x/pi}: divide by the pi bound that makes the
       quotient smaller (for qlo) or larger (for qhi) */
    double qlo = R_div(x.lo, x.lo >= 0.0 ? pi.hi : pi.lo, p, 0);
    double qhi = R_div(x.hi, x.hi >= 0.0 ? pi.lo : pi.hi, p, 1);
    if (!cos_not_sin) {            /* sin extrema at (k + 1/2) pi */
        qlo = R_sub(qlo, 0.5, p, 0);
        qhi = R_sub(qhi, 0.5, p, 1);
    }
    double k0 = ceil(qlo), k1 = floor(qhi);
    if (k0 <= k1) {
        int has_even = is_even(k0) || k0 + 1.0 <= k1;
        int has_odd = !is_even(k0) || k0 + 1.0 <= k1;
        if (has_even) hi = 1.0;    /* cos(2k pi) = 1, sin((2k+1/2) pi) = 1 */
        if (has_odd) lo = -1.0;
    }
    if (lo < -1.0) lo = -1.0;
    if (hi > 1.0) hi = 1.0;
    return mk(lo, hi);
}

/* ------------------------------------------------------------------------ */
/* Objective DAG (input format; 32-byte nodes)                               */
/* ------------------------------------------------------------------------ */
enum {
    O_CONST = 0, O_PI = 1, O_EULER = 2, O_VAR = 3, O_IDX_VAR = 4, O_IDX_COEF = 5,
    O_ADD = 6, O_SUB = 7, O_MUL = 8, O_DIV = 9, O_NEG = 10, O_SQR = 11,
    O_SQRT = 12, O_EXP = 13, O_SIN = 14, O_COS = 15, O_SCALE = 16, O_ISUM = 17,
    O_IPROD = 18, O_STEP = 19, O_COUNT = 20
};

/* ISUM and IPROD reduce a per-index template over an index set; they share
 * the layout, the grouping and the tree, and differ in the operation. */
static int is_red(int op) { return op == O_ISUM || op == O_IPROD; }

typedef struct { int32_t op, a, b, c, d, pad; double v; } onode;

static int n_operands(int op) {
    switch (op) {
    case O_ADD: case O_SUB: case O_MUL: case O_DIV: return 2;
    case O_NEG: case O_SQR: case O_SQRT: case O_EXP: case O_SIN: case O_COS:
    case O_SCALE: case O_STEP: return 1;
    default: return 0;
    }
}

typedef struct {
    int n, nn, root, B, nb;
    onode* nd;
    int ntab;
    double** tab;
    int64_t* tlen;
    double *l, *u;
    /* structure derived from the DAG */
    char* outer;          /* node reachable from root outside any template */
    char* in_tmpl;        /* scratch for template membership */
    int n_isum;           /* ISUM / IPROD nodes on the outer side, ascending */
    int* isum_node;
    int** tmpl_nodes;     /* per ISUM: template nodes ascending */
    int* tmpl_count;
    int* off_min;         /* per ISUM: min / max IDX_VAR offset */
    int* off_max;
    int* has_var;         /* per ISUM: template contains IDX_VAR */
    /* scratch */
    iv *val, *adj, *tval, *tadj, *terms, *groups, *gsum, *dacc, *gadj, *tseed;
    int* gstart;
    char* touched;
    int max_terms;
} oprob;

static int isum_count(const onode* s) {
    if (s->c <= s->b) return 0;
    return (s->c - s->b + s->d - 1) / s->d;
}

/* mark template nodes reachable from r into mark[]; fail on VAR / ISUM */
static int mark_template(const oprob* P, int r, char* mark) {
    if (mark[r]) return 0;
    mark[r] = 1;
    const onode* q = &P->nd[r];
    if (q->op == O_VAR || is_red(q->op)) return 1;
    int k = n_operands(q->op);
    if (k >= 1 && mark_template(P, q->a, mark)) return 1;
    if (k >= 2 && mark_template(P, q->b, mark)) return 1;
    return 0;
}

static int mark_outer(const oprob* P, int r) {
    if (P->outer[r]) return 0;
    P->outer[r] = 1;
    const onode* q = &P->nd[r];
    if (q->op == O_IDX_VAR || q->op == O_IDX_COEF) return 1;
    if (is_red(q->op)) return 0;             /* template handled separately */
    int k = n_operands(q->op);
    if (k >= 1 && mark_outer(P, q->a)) return 1;
    if (k >= 2 && mark_outer(P, q->b)) return 1;
    return 0;
}

static void free_prob(oprob* P) {
    if (!P) return;
    if (P->tab) for (int t = 0; t < P->ntab; t++) free(P->tab[t]);
    free(P->tab); free(P->tlen); free(P->nd); free(P->l); free(P->u);
    free(P->outer); free(P->in_tmpl); free(P->isum_node);
    if (P->tmpl_nodes) for (int k = 0; k < P->n_isum; k++) free(P->tmpl_nodes[k]);
    free(P->tmpl_nodes); free(P->tmpl_count); free(P->off_min); free(P->off_max);
    free(P->has_var);
    free(P->val); free(P->adj); free(P->tval); free(P->tadj); free(P->terms);
    free(P->groups); free(P->gsum); free(P->dacc); free(P->touched);
    free(P->gadj); free(P->tseed); free(P->gstart);
    free(P);
}

/* Copies and validates the problem (Eqs. 1-2: objective and simple bounds;
 * l < u finite).  Returns NULL on invalid input. */
static oprob* make_prob(const void* nodes, int nn, int root, const double* const* tables,
                        const int64_t* tlen, int ntab, int n, const double* l,
                        const double* u, int B) {
    init_constants();
    if (nn < 1 || root < 0 || root >= nn || n < 1 || ntab < 0 || B < 1 || B > n) return NULL;
    oprob* P = (oprob*)calloc(1, sizeof(oprob));
    P->n = n; P->nn = nn; P->root = root; P->B = B; P->nb = (n + B - 1) / B;
    P->nd = (onode*)malloc(sizeof(onode) * nn);
    memcpy(P->nd, nodes, sizeof(onode) * nn);
    P->ntab = ntab;
    P->tab = (double**)calloc(ntab > 0 ? ntab : 1, sizeof(double*));
    P->tlen = (int64_t*)calloc(ntab > 0 ? ntab : 1, sizeof(int64_t));
    for (int t = 0; t < ntab; t++) {
        if (tlen[t] < 0) { free_prob(P); return NULL; }
        P->tlen[t] = tlen[t];
        P->tab[t] = (double*)malloc(sizeof(double) * (tlen[t] > 0 ? tlen[t] : 1));
        memcpy(P->tab[t], tables[t], sizeof(double) * tlen[t]);
        for (int64_t i = 0; i < tlen[t]; i++)
            if (!isfinite(P->tab[t][i])) { free_prob(P); return NULL; }
    }
    P->l = (double*)malloc(sizeof(double) * n);
    P->u = (double*)malloc(sizeof(double) * n);
    for (int j = 0; j < n; j++) {
        P->l[j] = l[j]; P->u[j] = u[j];
        if (!isfinite(l[j]) || !isfinite(u[j]) || !(l[j] < u[j]) || !isfinite(u[j] - l[j])) {
            free_prob(P); return NULL;
        }
    }
    /* node-level checks: op range, topological operands */
    for (int v = 0; v < nn; v++) {
        const onode* q = &P->nd[v];
        if (q->op < 0 || q->op >= O_COUNT) { free_prob(P); return NULL; }
        int k = n_operands(q->op);
        if (k >= 1 && (q->a < 0 || q->a >= v)) { free_prob(P); return NULL; }
        if (k >= 2 && (q->b < 0 || q->b >= v)) { free_prob(P); return NULL; }
        if ((q->op == O_CONST || q->op == O_SCALE) && !isfinite(q->v)) { free_prob(P); return NULL; }
        if (q->op == O_VAR && (q->a < 0 || q->a >= n)) { free_prob(P); return NULL; }
        if (is_red(q->op) && (q->a < 0 || q->a >= v || q->d < 1)) { free_prob(P); return NULL; }
    }
    P->outer = (char*)calloc(nn, 1);
    P->in_tmpl = (char*)calloc(nn, 1);
    if (mark_outer(P, root)) { free_prob(P); return NULL; }
    /* ISUM / IPROD nodes and their templates */
    P->isum_node = (int*)malloc(sizeof(int) * nn);
    P->tmpl_nodes = (int**)calloc(nn, sizeof(int*));
    P->tmpl_count = (int*)calloc(nn, sizeof(int));
    P->off_min = (int*)calloc(nn, sizeof(int));
    P->off_max = (int*)calloc(nn, sizeof(int));
    P->has_var = (int*)calloc(nn, sizeof(int));
    int max_terms = 1;
    for (int v = 0; v < nn; v++) {
        if (!P->outer[v] || !is_red(P->nd[v].op)) continue;
        int k = P->n_isum++;
        P->isum_node[k] = v;
        const onode* s = &P->nd[v];
        memset(P->in_tmpl, 0, nn);
        if (mark_template(P, s->a, P->in_tmpl)) { free_prob(P); return NULL; }
        int cnt = 0;
        for (int t = 0; t <= s->a; t++) cnt += P->in_tmpl[t];
        P->tmpl_nodes[k] = (int*)malloc(sizeof(int) * cnt);
        P->tmpl_count[k] = cnt;
        cnt = 0;
        int omin = 0, omax = 0, hv = 0;
        for (int t = 0; t <= s->a; t++) {
            if (!P->in_tmpl[t]) continue;
            P->tmpl_nodes[k][cnt++] = t;
            if (P->nd[t].op == O_IDX_VAR) {
                int off = P->nd[t].b;
                if (!hv) { omin = omax = off; hv = 1; }
                if (off < omin) omin = off;
                if (off > omax) omax = off;
            }
        }
        P->off_min[k] = omin; P->off_max[k] = omax; P->has_var[k] = hv;
        int count = isum_count(s);
        if (count > max_terms) max_terms = count;
        if (count > 0) {
            int64_t ifirst = s->b, ilast = (int64_t)s->b + (int64_t)(count - 1) * s->d;
            if (hv && (ifirst + omin < 0 || ilast + omax >= n)) { free_prob(P); return NULL; }
            for (int t = 0; t < cnt; t++) {
                const onode* q = &P->nd[P->tmpl_nodes[k][t]];
                if (q->op == O_IDX_COEF) {
                    if (q->a < 0 || q->a >= ntab) { free_prob(P); return NULL; }
                    if (ifirst + q->b < 0 || ilast + q->b >= P->tlen[q->a]) { free_prob(P); return NULL; }
                }
            }
        }
    }
    P->max_terms = max_terms;
    P->val = (iv*)calloc(nn, sizeof(iv));
    P->adj = (iv*)calloc(nn, sizeof(iv));
    P->tval = (iv*)calloc(nn, sizeof(iv));
    P->tadj = (iv*)calloc(nn, sizeof(iv));
    P->terms = (iv*)calloc(max_terms, sizeof(iv));
    P->groups = (iv*)calloc(max_terms, sizeof(iv));
    P->gsum = (iv*)calloc(max_terms, sizeof(iv));
    P->gadj = (iv*)calloc(max_terms, sizeof(iv));
    P->tseed = (iv*)calloc(max_terms, sizeof(iv));
    P->gstart = (int*)calloc(max_terms + 1, sizeof(int));
    P->dacc = (iv*)calloc(B, sizeof(iv));
    P->touched = (char*)calloc(B, 1);
    return P;
}

/* A copy of P that shares its structure (read only) and owns fresh scratch
 * arrays, so that several threads can evaluate boxes of one problem. */
static oprob* clone_scratch(const oprob* P) {
    oprob* Q = (oprob*)malloc(sizeof(oprob));
    *Q = *P;
    Q->val = (iv*)calloc(P->nn, sizeof(iv));
    Q->adj = (iv*)calloc(P->nn, sizeof(iv));
    Q->tval = (iv*)calloc(P->nn, sizeof(iv));
    Q->tadj = (iv*)calloc(P->nn, sizeof(iv));
    Q->terms = (iv*)calloc(P->max_terms, sizeof(iv));
    Q->groups = (iv*)calloc(P->max_terms, sizeof(iv));
    Q->gsum = (iv*)calloc(P->max_terms, sizeof(iv));
    Q->gadj = (iv*)calloc(P->max_terms, sizeof(iv));
    Q->tseed = (iv*)calloc(P->max_terms, sizeof(iv));
    Q->gstart = (int*)calloc(P->max_terms + 1, sizeof(int));
    Q->dacc = (iv*)calloc(P->B, sizeof(iv));
    Q->touched = (char*)calloc(P->B, 1);
    return Q;
}

static void free_clone(oprob* Q) {
    if (!Q) return;
    free(Q->val); free(Q->adj); free(Q->tval); free(Q->tadj); free(Q->terms);
    free(Q->groups); free(Q->gsum); free(Q->gadj); free(Q->tseed); free(Q->gstart);
    free(Q->dacc); free(Q->touched);
    free(Q);
}

/* ------------------------------------------------------------------------ */
/* Evaluation                                                                */
/* ------------------------------------------------------------------------ */
typedef struct { const double *lo, *hi; } obox;

/* one node's forward value; i = ISUM index (templates), vals = value array */
static iv node_value(const oprob* P, int v, int i, obox X, int p, const iv* vals) {
    const onode* q = &P->nd[v];
    switch (q->op) {
    case O_CONST: return mk(R_in(q->v, p, 0), R_in(q->v, p, 1));
    case O_PI: return const_pi(p);
    case O_EULER: return const_e(p);
    case O_VAR: return mk(R_in(X.lo[q->a], p, 0), R_in(X.hi[q->a], p, 1));
    case O_IDX_VAR: return mk(R_in(X.lo[i + q->b], p, 0), R_in(X.hi[i + q->b], p, 1));
    case O_IDX_COEF: {
        double c = P->tab[q->a][i + q->b];
        return mk(R_in(c, p, 0), R_in(c, p, 1));
    }
    case O_ADD: return iv_add(vals[q->a], vals[q->b], p);
    case O_SUB: return iv_sub(vals[q->a], vals[q->b], p);
    case O_MUL: return iv_mul(vals[q->a], vals[q->b], p);
    case O_DIV: return iv_div(vals[q->a], vals[q->b], p);
    case O_NEG: return iv_neg(vals[q->a]);
    case O_SQR: return iv_sqr(vals[q->a], p);
    case O_SQRT: return iv_sqrt(vals[q->a], p);
    case O_EXP: return iv_exp(vals[q->a], p);
    case O_SIN: return iv_trig(vals[q->a], p, 0);
    case O_COS: return iv_trig(vals[q->a], p, 1);
    case O_SCALE: return iv_scale(vals[q->a], q->v, p);
    case O_STEP: return iv_step(vals[q->a]);
    default: return entire();
    }
}

/* Reverse-mode step: adds node v's contributions to its operands' adjoints
 * (first operand a, then b).  Because v runs from high to low index, each
 * adjoint receives its consumers' contributions in descending consumer order,
 * starting from [0, 0].  The derivative formulas are the natural interval
 * extensions of d(op)/d(operand). */
static void push_adjoint(const oprob* P, int v, int p, const iv* vals, iv* adj) {
    const onode* q = &P->nd[v];
    iv g = adj[v];
    switch (q->op) {
    case O_ADD:
        adj[q->a] = iv_add(adj[q->a], g, p);
        adj[q->b] = iv_add(adj[q->b], g, p);
        break;
    case O_SUB:
        adj[q->a] = iv_add(adj[q->a], g, p);
        adj[q->b] = iv_add(adj[q->b], iv_neg(g), p);
        break;
    case O_MUL:
        adj[q->a] = iv_add(adj[q->a], iv_mul(g, vals[q->b], p), p);
        adj[q->b] = iv_add(adj[q->b], iv_mul(g, vals[q->a], p), p);
        break;
    case O_DIV: {
        iv rb = iv_recip(vals[q->b], p);
        adj[q->a] = iv_add(adj[q->a], iv_mul(g, rb, p), p);
        adj[q->b] = iv_add(adj[q->b], iv_mul(g, iv_neg(iv_mul(vals[v], rb, p)), p), p);
        break;
    }
    case O_NEG:
        adj[q->a] = iv_add(adj[q->a], iv_neg(g), p);
        break;
    case O_SQR:
        adj[q->a] = iv_add(adj[q->a], iv_mul(g, iv_scale(vals[q->a], 2.0, p), p), p);
        break;
    case O_SQRT:
        adj[q->a] = iv_add(adj[q->a], iv_mul(g, iv_scale(iv_recip(vals[v], p), 0.5, p), p), p);
        break;
    case O_EXP:
        adj[q->a] = iv_add(adj[q->a], iv_mul(g, vals[v], p), p);
        break;
    case O_SIN:
        adj[q->a] = iv_add(adj[q->a], iv_mul(g, iv_trig(vals[q->a], p, 1), p), p);
        break;
    case O_COS:
        adj[q->a] = iv_add(adj[q->a], iv_mul(g, iv_neg(iv_trig(vals[q->a], p, 0)), p), p);
        break;
    case O_SCALE:
        adj[q->a] = iv_add(adj[q->a], iv_scale(g, q->v, p), p);
        break;
    case O_STEP:
        /* H' = 0 off the jump; a box that holds the jump (with a nonzero
         * adjoint) gets an unbounded partial, so the first-order test keeps it.
         * Reading: the paper gives no rule for partials of a discontinuous f. */
        if (step_jump(vals[q->a]) && !(g.lo == 0.0 && g.hi == 0.0))
            adj[q->a] = iv_add(adj[q->a], entire(), p);
        break;
    default:
        break;
    }
}

/* Pairwise reduction tree over a[0..m) in index order, in place:
 * level s = 1, 2, 4, ...: a[i] += a[i + s] for i = 0, 2s, 4s, ... while
 * i + s < m.  Reading: the paper does not fix a summation order; this one is
 * fixed so that every implementation produces the same bits. */
static iv tree_sum(iv* a, int m, int p) {
    if (m == 0) return mk(0.0, 0.0);
    for (int s = 1; s < m; s *= 2)
        for (int i = 0; i + s < m; i += 2 * s) a[i] = iv_add(a[i], a[i + s], p);
    return a[0];
}

/* The same tree with products (IPROD); the empty product is [1, 1]. */
static iv tree_prod(iv* a, int m, int p) {
    if (m == 0) return mk(1.0, 1.0);
    for (int s = 1; s < m; s *= 2)
        for (int i = 0; i + s < m; i += 2 * s) a[i] = iv_mul(a[i], a[i + s], p);
    return a[0];
}

/* Reverse sweep of tree_prod over a[0..m): adj[i] receives the adjoint of
 * item i when the product has adjoint seed.  Every tree node feeds exactly
 * one product, so a node's adjoint is its consumer's adjoint times the other
 * operand's value (reverse mode over the tree's code list, top level first).
 * Reading: the paper does not say how partials are formed (section 3.1);
 * this is the reverse-mode rule of every other operation applied to the
 * fixed reduction tree. */
static void tree_prod_adjoint(const iv* a, int m, iv seed, iv* adj, int p) {
    if (m == 0) return;
    int L = 0;
    while ((1 << L) < m) L++;
    iv* V = (iv*)malloc(sizeof(iv) * (size_t)m * (L + 1));   /* values entering level l */
    iv* A = (iv*)malloc(sizeof(iv) * (size_t)m * (L + 1));   /* their adjoints */
    memcpy(V, a, sizeof(iv) * (size_t)m);
    for (int l = 0; l < L; l++) {
        const int s = 1 << l;
        const iv* cur = V + (size_t)l * m;
        iv* nxt = V + (size_t)(l + 1) * m;
        memcpy(nxt, cur, sizeof(iv) * (size_t)m);
        for (int i = 0; i + s < m; i += 2 * s) nxt[i] = iv_mul(cur[i], cur[i + s], p);
    }
    A[(size_t)L * m] = seed;
    for (int l = L - 1; l >= 0; l--) {
        const int s = 1 << l;
        const iv* cur = V + (size_t)l * m;
        const iv* up = A + (size_t)(l + 1) * m;
        iv* dn = A + (size_t)l * m;
        for (int i = 0; i < m; i += 2 * s) {
            if (i + s < m) {
                dn[i] = iv_mul(up[i], cur[i + s], p);
                dn[i + s] = iv_mul(up[i], cur[i], p);
            } else {
                dn[i] = up[i];
            }
        }
    }
    memcpy(adj, A, sizeof(iv) * (size_t)m);
    free(V);
    free(A);
}

/* Evaluates template k (ISUM node index isum_node[k]) for index i; values
 * in P->tval, returns the root value. */
static iv eval_term(oprob* P, int k, int i, obox X, int p) {
    for (int t = 0; t < P->tmpl_count[k]; t++) {
        int v = P->tmpl_nodes[k][t];
        P->tval[v] = node_value(P, v, i, X, p, P->tval);
    }
    return P->tval[P->nd[P->isum_node[k]].a];
}

/* Block range [bmin, bmax] of the coordinates term i of ISUM k touches. */
static void term_blocks(const oprob* P, int k, int i, int* bmin, int* bmax) {
    if (!P->has_var[k]) { *bmin = *bmax = -1; return; }
    *bmin = (i + P->off_min[k]) / P->B;
    *bmax = (i + P->off_max[k]) / P->B;
}

/* Groups of reduction k: terms in index order split into maximal runs with
 * the same touched-block range; group g holds the term ordinals
 * [gstart[g], gstart[g + 1]).  Returns the number of groups. */
static int isum_groups(const oprob* P, int k, int* gstart) {
    const onode* s = &P->nd[P->isum_node[k]];
    int cnt = isum_count(s);
    int ng = 0, start = 0;
    if (cnt == 0) return 0;
    for (int q = 1; q <= cnt; q++) {
        int b0, b1, c0, c1;
        term_blocks(P, k, s->b + start * s->d, &b0, &b1);
        int boundary = (q == cnt);
        if (!boundary) {
            term_blocks(P, k, s->b + q * s->d, &c0, &c1);
            boundary = (c0 != b0 || c1 != b1);
        }
        if (boundary) {
            gstart[ng++] = start;
            start = q;
        }
    }
    gstart[ng] = cnt;
    return ng;
}

/* ISUM / IPROD value: each group reduced by the tree (sum or product),
 * then the groups in order by the tree again.  Leaves the term values in
 * P->terms and the group values in P->gsum. */
static iv isum_value(oprob* P, int k, obox X, int p) {
    const onode* s = &P->nd[P->isum_node[k]];
    const int prod = s->op == O_IPROD;
    int cnt = isum_count(s);
    if (cnt == 0) return prod ? mk(1.0, 1.0) : mk(0.0, 0.0);
    for (int q = 0; q < cnt; q++) P->terms[q] = eval_term(P, k, s->b + q * s->d, X, p);
    int ng = isum_groups(P, k, P->gstart);
    for (int g = 0; g < ng; g++) {
        int a = P->gstart[g], e = P->gstart[g + 1];
        for (int r = a; r < e; r++) P->groups[r - a] = P->terms[r];
        P->gsum[g] = prod ? tree_prod(P->groups, e - a, p) : tree_sum(P->groups, e - a, p);
    }
    for (int g = 0; g < ng; g++) P->groups[g] = P->gsum[g];
    return prod ? tree_prod(P->groups, ng, p) : tree_sum(P->groups, ng, p);
}

/* Forward pass of the outer expression; returns F(X). */
static iv eval_outer(oprob* P, obox X, int p) {
    int k = 0;
    for (int v = 0; v < P->nn; v++) {
        if (!P->outer[v]) continue;
        if (is_red(P->nd[v].op)) {
            while (P->isum_node[k] != v) k++;
            P->val[v] = isum_value(P, k, X, p);
        } else {
            P->val[v] = node_value(P, v, -1, X, p, P->val);
        }
    }
    return P->val[P->root];
}

/* Interval partials of f for the coordinates of block blk (section 3.1's
 * first-order test needs [DLB_i, DUB_i]).  Reading: reverse-mode interval
 * adjoints; for coordinate j the sum runs over the outer VAR(j) leaves
 * (ascending node), then over the ISUM / IPROD nodes (ascending) of
 * adj(node) * D_j, where D_j sums the template adjoints of the IDX_VAR leaves
 * that hit x_j, in ascending term index and ascending leaf node.  A sum's
 * templates are seeded with [1,1]; a product's with the term's adjoint in
 * the product tree (tree_prod_adjoint, seed [1,1]).  Requires eval_outer(X)
 * to have run.  G has B entries. */
static void block_partials(oprob* P, obox X, int p, int blk, iv* G, int* width) {
    int c0 = blk * P->B, c1 = c0 + P->B;
    if (c1 > P->n) c1 = P->n;
    *width = c1 - c0;
    for (int v = 0; v < P->nn; v++) P->adj[v] = mk(0.0, 0.0);
    P->adj[P->root] = mk(1.0, 1.0);
    for (int v = P->nn - 1; v >= 0; v--) {
        if (!P->outer[v] || is_red(P->nd[v].op)) continue;
        push_adjoint(P, v, p, P->val, P->adj);
    }
    for (int j = c0; j < c1; j++) G[j - c0] = mk(0.0, 0.0);
    for (int v = 0; v < P->nn; v++)
        if (P->outer[v] && P->nd[v].op == O_VAR && P->nd[v].a >= c0 && P->nd[v].a < c1)
            G[P->nd[v].a - c0] = iv_add(G[P->nd[v].a - c0], P->adj[v], p);
    for (int k = 0; k < P->n_isum; k++) {
        if (!P->has_var[k]) continue;
        const onode* s = &P->nd[P->isum_node[k]];
        int cnt = isum_count(s);
        const int prod = s->op == O_IPROD;
        if (prod) {
            /* a term's adjoint within the product (seed [1, 1] at the
             * product): the group tree's reverse sweep, then the group's */
            isum_value(P, k, X, p);
            int ng = isum_groups(P, k, P->gstart);
            tree_prod_adjoint(P->gsum, ng, mk(1.0, 1.0), P->gadj, p);
            for (int g = 0; g < ng; g++)
                tree_prod_adjoint(P->terms + P->gstart[g], P->gstart[g + 1] - P->gstart[g], P->gadj[g],
                                  P->tseed + P->gstart[g], p);
        }
        for (int j = c0; j < c1; j++) { P->dacc[j - c0] = mk(0.0, 0.0); P->touched[j - c0] = 0; }
        for (int q = 0; q < cnt; q++) {
            int i = s->b + q * s->d;
            if (i + P->off_max[k] < c0 || i + P->off_min[k] >= c1) continue;
            eval_term(P, k, i, X, p);
            int troot = s->a;
            for (int t = 0; t < P->tmpl_count[k]; t++) P->tadj[P->tmpl_nodes[k][t]] = mk(0.0, 0.0);
            P->tadj[troot] = prod ? P->tseed[q] : mk(1.0, 1.0);
            for (int t = P->tmpl_count[k] - 1; t >= 0; t--)
                push_adjoint(P, P->tmpl_nodes[k][t], p, P->tval, P->tadj);
            for (int t = 0; t < P->tmpl_count[k]; t++) {
                const onode* leaf = &P->nd[P->tmpl_nodes[k][t]];
                if (leaf->op != O_IDX_VAR) continue;
                int j = i + leaf->b;
                if (j < c0 || j >= c1) continue;
                P->dacc[j - c0] = iv_add(P->dacc[j - c0], P->tadj[P->tmpl_nodes[k][t]], p);
                P->touched[j - c0] = 1;
            }
        }
        for (int j = c0; j < c1; j++)
            if (P->touched[j - c0])
                G[j - c0] = iv_add(G[j - c0], iv_mul(P->adj[P->isum_node[k]], P->dacc[j - c0], p), p);
    }
}

/* First-order test of section 3.1: the box is ruled out if some tested
 * partial has DLB > 0 while its lower face is not on l, or DUB < 0 while
 * its upper face is not on u.  Reading: the tested coordinates are those of
 * the box's active cycling block. */
static int mono_test(const oprob* P, obox X, int blk, const iv* G, int width) {
    int c0 = blk * P->B;
    for (int t = 0; t < width; t++) {
        int j = c0 + t;
        if (G[t].lo > 0.0 && X.lo[j] != P->l[j]) return 1;
        if (G[t].hi < 0.0 && X.hi[j] != P->u[j]) return 1;
    }
    return 0;
}

/* Midpoint sample point (section 3.1 allows any sampling strategy; reading:
 * one point per box, mid = RN(0.5 lo + 0.5 hi)). */
static double midpoint(double lo, double hi) {
    volatile double a = 0.5 * lo;
    volatile double b = 0.5 * hi;
    return a + b;
}

static double canon_lo(double x) {
    if (isnan(x)) return -INFINITY;
    if (x == 0.0) return 0.0;
    return x;
}

static uint64_t order_key(double x) {
    uint64_t b;
    memcpy(&b, &x, 8);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

/* ------------------------------------------------------------------------ */
/* Deviation bound (the tolerance of transcendental parity)                  */
/* ------------------------------------------------------------------------ */
/* Two implementations that run the same directed operations in the same
 * order produce the same bits; they can differ only where a library
 * transcendental (exp, sin, cos) is called, because each library is only
 * within its documented error of the true value and each side widens by its
 * own count of ulps.  Beside every interval the oracle computes, the
 * functions below carry a number d >= 0 such that an implementation whose
 * transcendental endpoints lie within DEV_KT ulps of the oracle's produces
 * endpoints (both ends) within d of the oracle's.  Rules (first order plus
 * the second-order terms, all rounded upward; mag = larger endpoint
 * magnitude):
 *   constants, coordinates, coefficients     d = 0
 *   a + b, a - b                             da + db
 *   a * b (min / max of products)            mag(b) da + mag(a) db + da db
 *   1 / b                                    db / (mig(b) (mig(b) - db)); infinite when db >= mig(b)
 *   a^2                                      (2 mag(a) + da) da
 *   sqrt(a)                                  min(sqrt(da), da / (2 sqrt(lo(a) - da)))
 *   exp(a)                                   KT ulp(mag) + exp(hi(a) + da) da
 *   sin(a), cos(a)                           KT ulp(mag) + da + (2 ulp(mag a) + 2 da)^2
 *                                            (the last term covers an extremum that one side
 *                                            includes and the other does not); 2 when the width
 *                                            test may decide differently
 *   unit step                                1 when a lies within da of the jump, else 0
 * and every rounded result whose operands deviate gains one ulp (directed
 * rounding of two different exact values differs by at most their distance
 * plus one ulp).  Reading of the "width within 4 ulp n" requirement for
 * transcendental families: the GPU result must lie within d of the oracle's;
 * for objectives without transcendentals d = 0 (bit-exact parity). */
#define DEV_KT 8.0

static double up_add(double a, double b) { return d_add(a, b, 1); }
static double umul(double a, double b) { return (a == 0.0 || b == 0.0) ? 0.0 : d_mul(a, b, 1); }
static double magv(iv x) {
    double m = fmax(fabs(x.lo), fabs(x.hi));
    return isnan(x.lo) || isnan(x.hi) ? INFINITY : m;
}
/* Twice the spacing of precision p at magnitude m: one ulp of any value up
 * to just past the next power of two. */
static double ulp_at(double m, int p) {
    m = fabs(m);
    if (!(m < INFINITY)) return INFINITY;
    if (p) {
        float f = (float)m;
        if ((double)f < m) f = nextafterf(f, INFINITY);
        return 2.0 * ((double)nextafterf(f, INFINITY) - (double)f);
    }
    return 2.0 * (nextafter(m, INFINITY) - m);
}
static double dflip(double d, iv r, int p) { return d > 0.0 ? up_add(d, ulp_at(magv(r), p)) : 0.0; }

static double dev_mul(iv a, double da, iv b, double db) {
    return up_add(up_add(umul(magv(b), da), umul(magv(a), db)), umul(da, db));
}
static double mig(iv y) { return y.lo > 0.0 ? y.lo : (y.hi < 0.0 ? -y.hi : 0.0); }
static double dev_recip(iv y, double dy, iv r, int p) {
    if (dy == 0.0) return 0.0;
    double m = mig(y);
    if (!(m > dy)) return INFINITY;
    return dflip(d_div(dy, d_mul(m, d_sub(m, dy, 0), 0), 1), r, p);
}
static double dev_sqrt(iv a, double da, iv r, int p) {
    if (da == 0.0) return 0.0;
    double d = d_sqrt(da, 1);
    double m = d_sub(a.lo, da, 0);
    if (m > 0.0) d = fmin(d, d_div(da, d_mul(2.0, d_sqrt(m, 0), 0), 1));
    return dflip(d, r, p);
}
static double dev_exp(iv a, double da, iv r, int p) {
    double d = DEV_KT * ulp_at(magv(r), p);
    if (da > 0.0) {
        double e = nextafter(nextafter(exp(up_add(a.hi, da)), INFINITY), INFINITY);
        d = up_add(d, dflip(umul(e, da), r, p));
    }
    return d;
}
static double dev_trig(iv a, double da, iv r, int p) {
    double d = DEV_KT * ulp_at(magv(r), p);
    if (da == 0.0) return d;
    double big = p ? 1048576.0 : 1099511627776.0;
    double w = up_add(up_add(d_sub(a.hi, a.lo, 1), da), da);
    if (!(w < 2.0 * PI_LO) || !(up_add(magv(a), da) <= big)) return 2.0;
    double e = up_add(ulp_at(magv(a), p), up_add(da, da));
    return dflip(up_add(up_add(d, da), umul(e, e)), r, p);
}
static double scale_mag(double c, int p) {
    return p ? fmax(fabs(R_in(c, 1, 0)), fabs(R_in(c, 1, 1))) : fabs(c);
}

/* Deviation of node v's value r from its operands' values and deviations. */
static double node_dev(const oprob* P, int v, int p, const iv* vals, const double* devs, iv r) {
    const onode* q = &P->nd[v];
    const int k = n_operands(q->op);
    iv a = mk(0.0, 0.0), b = mk(0.0, 0.0);
    double da = 0.0, db = 0.0;
    if (k >= 1) { a = vals[q->a]; da = devs[q->a]; }
    if (k >= 2) { b = vals[q->b]; db = devs[q->b]; }
    switch (q->op) {
    case O_ADD: case O_SUB: return dflip(up_add(da, db), r, p);
    case O_MUL: return dflip(dev_mul(a, da, b, db), r, p);
    case O_DIV: {
        iv rb = iv_recip(b, p);
        return dflip(dev_mul(a, da, rb, dev_recip(b, db, rb, p)), r, p);
    }
    case O_NEG: return da;
    case O_SQR: return dflip(umul(up_add(umul(2.0, magv(a)), da), da), r, p);
    case O_SQRT: return dev_sqrt(a, da, r, p);
    case O_EXP: return dev_exp(a, da, r, p);
    case O_SIN: case O_COS: return dev_trig(a, da, r, p);
    case O_SCALE: return dflip(umul(scale_mag(q->v, p), da), r, p);
    case O_STEP: return (da > 0.0 && (fabs(a.lo) <= da || fabs(a.hi) <= da)) ? 1.0 : 0.0;
    default: return 0.0;
    }
}

/* The reduction trees with deviations carried beside the values. */
static void tree_dev(iv* a, double* d, int m, int p, int prod) {
    for (int s = 1; s < m; s *= 2)
        for (int i = 0; i + s < m; i += 2 * s) {
            iv r = prod ? iv_mul(a[i], a[i + s], p) : iv_add(a[i], a[i + s], p);
            d[i] = dflip(prod ? dev_mul(a[i], d[i], a[i + s], d[i + s]) : up_add(d[i], d[i + s]), r, p);
            a[i] = r;
        }
}

/* tree_prod_adjoint with deviations: adj / dadj receive each item's adjoint. */
static void tree_prod_adjoint_dev(const iv* a, const double* da, int m, iv seed, double dseed, iv* adj,
                                  double* dadj, int p) {
    if (m == 0) return;
    int L = 0;
    while ((1 << L) < m) L++;
    const size_t sz = (size_t)m * (L + 1);
    iv* V = (iv*)malloc(sizeof(iv) * sz);
    iv* A = (iv*)malloc(sizeof(iv) * sz);
    double* DV = (double*)malloc(sizeof(double) * sz);
    double* DA = (double*)malloc(sizeof(double) * sz);
    memcpy(V, a, sizeof(iv) * (size_t)m);
    memcpy(DV, da, sizeof(double) * (size_t)m);
    for (int l = 0; l < L; l++) {
        const int s = 1 << l;
        const size_t c = (size_t)l * m, nx = (size_t)(l + 1) * m;
        memcpy(V + nx, V + c, sizeof(iv) * (size_t)m);
        memcpy(DV + nx, DV + c, sizeof(double) * (size_t)m);
        for (int i = 0; i + s < m; i += 2 * s) {
            V[nx + i] = iv_mul(V[c + i], V[c + i + s], p);
            DV[nx + i] = dflip(dev_mul(V[c + i], DV[c + i], V[c + i + s], DV[c + i + s]), V[nx + i], p);
        }
    }
    A[(size_t)L * m] = seed;
    DA[(size_t)L * m] = dseed;
    for (int l = L - 1; l >= 0; l--) {
        const int s = 1 << l;
        const size_t c = (size_t)l * m, up = (size_t)(l + 1) * m;
        for (int i = 0; i < m; i += 2 * s) {
            if (i + s < m) {
                A[c + i] = iv_mul(A[up + i], V[c + i + s], p);
                DA[c + i] = dflip(dev_mul(A[up + i], DA[up + i], V[c + i + s], DV[c + i + s]), A[c + i], p);
                A[c + i + s] = iv_mul(A[up + i], V[c + i], p);
                DA[c + i + s] = dflip(dev_mul(A[up + i], DA[up + i], V[c + i], DV[c + i]), A[c + i + s], p);
            } else {
                A[c + i] = A[up + i];
                DA[c + i] = DA[up + i];
            }
        }
    }
    memcpy(adj, A, sizeof(iv) * (size_t)m);
    memcpy(dadj, DA, sizeof(double) * (size_t)m);
    free(V); free(A); free(DV); free(DA);
}

/* Scratch of one deviation evaluation (values beside their deviations). */
typedef struct {
    iv *val, *adj, *tval, *tadj, *terms, *grp, *gsum, *gadj, *tseed, *dacc, *G;
    double *dval, *dadj, *dtval, *dtadj, *dterms, *dgrp, *dgsum, *dgadj, *dtseed, *ddacc, *dG;
    int* gstart;
    char* touched;
} dscr;

static void dscr_alloc(const oprob* P, dscr* S) {
    const size_t nn = (size_t)P->nn, mt = (size_t)P->max_terms, B = (size_t)P->B;
    S->val = (iv*)calloc(nn, sizeof(iv)); S->dval = (double*)calloc(nn, sizeof(double));
    S->adj = (iv*)calloc(nn, sizeof(iv)); S->dadj = (double*)calloc(nn, sizeof(double));
    S->tval = (iv*)calloc(nn, sizeof(iv)); S->dtval = (double*)calloc(nn, sizeof(double));
    S->tadj = (iv*)calloc(nn, sizeof(iv)); S->dtadj = (double*)calloc(nn, sizeof(double));
    S->terms = (iv*)calloc(mt, sizeof(iv)); S->dterms = (double*)calloc(mt, sizeof(double));
    S->grp = (iv*)calloc(mt, sizeof(iv)); S->dgrp = (double*)calloc(mt, sizeof(double));
    S->gsum = (iv*)calloc(mt, sizeof(iv)); S->dgsum = (double*)calloc(mt, sizeof(double));
    S->gadj = (iv*)calloc(mt, sizeof(iv)); S->dgadj = (double*)calloc(mt, sizeof(double));
    S->tseed = (iv*)calloc(mt, sizeof(iv)); S->dtseed = (double*)calloc(mt, sizeof(double));
    S->dacc = (iv*)calloc(B, sizeof(iv)); S->ddacc = (double*)calloc(B, sizeof(double));
    S->G = (iv*)calloc(B, sizeof(iv)); S->dG = (double*)calloc(B, sizeof(double));
    S->gstart = (int*)calloc(mt + 1, sizeof(int));
    S->touched = (char*)calloc(B, 1);
}

static void dscr_free(dscr* S) {
    free(S->val); free(S->dval); free(S->adj); free(S->dadj); free(S->tval); free(S->dtval);
    free(S->tadj); free(S->dtadj); free(S->terms); free(S->dterms); free(S->grp); free(S->dgrp);
    free(S->gsum); free(S->dgsum); free(S->gadj); free(S->dgadj); free(S->tseed); free(S->dtseed);
    free(S->dacc); free(S->ddacc); free(S->G); free(S->dG); free(S->gstart); free(S->touched);
}

/* Template k at index i: values in S->tval, deviations in S->dtval. */
static void dev_term(const oprob* P, int k, int i, obox X, int p, dscr* S) {
    for (int t = 0; t < P->tmpl_count[k]; t++) {
        int v = P->tmpl_nodes[k][t];
        S->tval[v] = node_value(P, v, i, X, p, S->tval);
        S->dtval[v] = node_dev(P, v, p, S->tval, S->dtval, S->tval[v]);
    }
}

/* Reduction k with deviations (isum_value's groups and trees); leaves the
 * term values in S->terms and the group values in S->gsum. */
static iv dev_reduction(const oprob* P, int k, obox X, int p, dscr* S, double* d) {
    const onode* s = &P->nd[P->isum_node[k]];
    const int prod = s->op == O_IPROD;
    int cnt = isum_count(s);
    if (cnt == 0) { *d = 0.0; return prod ? mk(1.0, 1.0) : mk(0.0, 0.0); }
    for (int q = 0; q < cnt; q++) {
        dev_term(P, k, s->b + q * s->d, X, p, S);
        S->terms[q] = S->tval[s->a];
        S->dterms[q] = S->dtval[s->a];
    }
    int ng = isum_groups(P, k, S->gstart);
    for (int g = 0; g < ng; g++) {
        int a = S->gstart[g], e = S->gstart[g + 1];
        for (int r = a; r < e; r++) { S->grp[r - a] = S->terms[r]; S->dgrp[r - a] = S->dterms[r]; }
        tree_dev(S->grp, S->dgrp, e - a, p, prod);
        S->gsum[g] = S->grp[0];
        S->dgsum[g] = S->dgrp[0];
    }
    for (int g = 0; g < ng; g++) { S->grp[g] = S->gsum[g]; S->dgrp[g] = S->dgsum[g]; }
    tree_dev(S->grp, S->dgrp, ng, p, prod);
    *d = S->dgrp[0];
    return S->grp[0];
}

/* Forward pass of the outer expression with deviations. */
static iv dev_outer(const oprob* P, obox X, int p, dscr* S, double* d) {
    int k = 0;
    for (int v = 0; v < P->nn; v++) {
        if (!P->outer[v]) continue;
        if (is_red(P->nd[v].op)) {
            while (P->isum_node[k] != v) k++;
            S->val[v] = dev_reduction(P, k, X, p, S, &S->dval[v]);
        } else {
            S->val[v] = node_value(P, v, -1, X, p, S->val);
            S->dval[v] = node_dev(P, v, p, S->val, S->dval, S->val[v]);
        }
    }
    *d = S->dval[P->root];
    return S->val[P->root];
}

/* adj[t] += x with deviations. */
static void acc_dev(iv* adj, double* dadj, int t, iv x, double dx, int p) {
    iv r = iv_add(adj[t], x, p);
    dadj[t] = dflip(up_add(dadj[t], dx), r, p);
    adj[t] = r;
}

/* push_adjoint with deviations. */
static void push_adjoint_dev(const oprob* P, int v, int p, const iv* vals, const double* dv, iv* adj,
                             double* dadj) {
    const onode* q = &P->nd[v];
    const iv g = adj[v];
    const double dg = dadj[v];
    iv x;
    switch (q->op) {
    case O_ADD:
        acc_dev(adj, dadj, q->a, g, dg, p);
        acc_dev(adj, dadj, q->b, g, dg, p);
        break;
    case O_SUB:
        acc_dev(adj, dadj, q->a, g, dg, p);
        acc_dev(adj, dadj, q->b, iv_neg(g), dg, p);
        break;
    case O_MUL:
        x = iv_mul(g, vals[q->b], p);
        acc_dev(adj, dadj, q->a, x, dflip(dev_mul(g, dg, vals[q->b], dv[q->b]), x, p), p);
        x = iv_mul(g, vals[q->a], p);
        acc_dev(adj, dadj, q->b, x, dflip(dev_mul(g, dg, vals[q->a], dv[q->a]), x, p), p);
        break;
    case O_DIV: {
        iv rb = iv_recip(vals[q->b], p);
        double drb = dev_recip(vals[q->b], dv[q->b], rb, p);
        x = iv_mul(g, rb, p);
        acc_dev(adj, dadj, q->a, x, dflip(dev_mul(g, dg, rb, drb), x, p), p);
        iv y = iv_mul(vals[v], rb, p);
        double dy = dflip(dev_mul(vals[v], dv[v], rb, drb), y, p);
        x = iv_mul(g, iv_neg(y), p);
        acc_dev(adj, dadj, q->b, x, dflip(dev_mul(g, dg, y, dy), x, p), p);
        break;
    }
    case O_NEG:
        acc_dev(adj, dadj, q->a, iv_neg(g), dg, p);
        break;
    case O_SQR: {
        iv s2 = iv_scale(vals[q->a], 2.0, p);
        double ds2 = dflip(umul(2.0, dv[q->a]), s2, p);
        x = iv_mul(g, s2, p);
        acc_dev(adj, dadj, q->a, x, dflip(dev_mul(g, dg, s2, ds2), x, p), p);
        break;
    }
    case O_SQRT: {
        iv rv = iv_recip(vals[v], p);
        double drv = dev_recip(vals[v], dv[v], rv, p);
        iv h = iv_scale(rv, 0.5, p);
        double dh = dflip(umul(0.5, drv), h, p);
        x = iv_mul(g, h, p);
        acc_dev(adj, dadj, q->a, x, dflip(dev_mul(g, dg, h, dh), x, p), p);
        break;
    }
    case O_EXP:
        x = iv_mul(g, vals[v], p);
        acc_dev(adj, dadj, q->a, x, dflip(dev_mul(g, dg, vals[v], dv[v]), x, p), p);
        break;
    case O_SIN: case O_COS: {
        iv c = iv_trig(vals[q->a], p, q->op == O_SIN);
        double dc = dev_trig(vals[q->a], dv[q->a], c, p);
        if (q->op == O_COS) c = iv_neg(c);
        x = iv_mul(g, c, p);
        acc_dev(adj, dadj, q->a, x, dflip(dev_mul(g, dg, c, dc), x, p), p);
        break;
    }
    case O_SCALE:
        x = iv_scale(g, q->v, p);
        acc_dev(adj, dadj, q->a, x, dflip(umul(scale_mag(q->v, p), dg), x, p), p);
        break;
    case O_STEP: {
        const iv a = vals[q->a];
        const double da = dv[q->a];
        const int unsure = (da > 0.0 && (fabs(a.lo) <= da || fabs(a.hi) <= da)) ||
                           (dg > 0.0 && fabs(g.lo) <= dg && fabs(g.hi) <= dg);
        if (step_jump(a) && !(g.lo == 0.0 && g.hi == 0.0)) acc_dev(adj, dadj, q->a, entire(), 0.0, p);
        if (unsure) dadj[q->a] = INFINITY;
        break;
    }
    default:
        break;
    }
}

/* block_partials with deviations: S->G[0..width) and S->dG.  Needs
 * dev_outer(X) to have run on S. */
static void dev_block_partials(const oprob* P, obox X, int p, int blk, dscr* S, int* width) {
    int c0 = blk * P->B, c1 = c0 + P->B;
    if (c1 > P->n) c1 = P->n;
    *width = c1 - c0;
    for (int v = 0; v < P->nn; v++) { S->adj[v] = mk(0.0, 0.0); S->dadj[v] = 0.0; }
    S->adj[P->root] = mk(1.0, 1.0);
    for (int v = P->nn - 1; v >= 0; v--) {
        if (!P->outer[v] || is_red(P->nd[v].op)) continue;
        push_adjoint_dev(P, v, p, S->val, S->dval, S->adj, S->dadj);
    }
    for (int j = c0; j < c1; j++) { S->G[j - c0] = mk(0.0, 0.0); S->dG[j - c0] = 0.0; }
    for (int v = 0; v < P->nn; v++)
        if (P->outer[v] && P->nd[v].op == O_VAR && P->nd[v].a >= c0 && P->nd[v].a < c1)
            acc_dev(S->G, S->dG, P->nd[v].a - c0, S->adj[v], S->dadj[v], p);
    for (int k = 0; k < P->n_isum; k++) {
        if (!P->has_var[k]) continue;
        const onode* s = &P->nd[P->isum_node[k]];
        int cnt = isum_count(s);
        const int prod = s->op == O_IPROD;
        if (prod) {
            double dd;
            dev_reduction(P, k, X, p, S, &dd);
            int ng = isum_groups(P, k, S->gstart);
            tree_prod_adjoint_dev(S->gsum, S->dgsum, ng, mk(1.0, 1.0), 0.0, S->gadj, S->dgadj, p);
            for (int g = 0; g < ng; g++)
                tree_prod_adjoint_dev(S->terms + S->gstart[g], S->dterms + S->gstart[g],
                                      S->gstart[g + 1] - S->gstart[g], S->gadj[g], S->dgadj[g],
                                      S->tseed + S->gstart[g], S->dtseed + S->gstart[g], p);
        }
        for (int j = c0; j < c1; j++) { S->dacc[j - c0] = mk(0.0, 0.0); S->ddacc[j - c0] = 0.0; S->touched[j - c0] = 0; }
        for (int q = 0; q < cnt; q++) {
            int i = s->b + q * s->d;
            if (i + P->off_max[k] < c0 || i + P->off_min[k] >= c1) continue;
            dev_term(P, k, i, X, p, S);
            int troot = s->a;
            for (int t = 0; t < P->tmpl_count[k]; t++) {
                S->tadj[P->tmpl_nodes[k][t]] = mk(0.0, 0.0);
                S->dtadj[P->tmpl_nodes[k][t]] = 0.0;
            }
            S->tadj[troot] = prod ? S->tseed[q] : mk(1.0, 1.0);
            S->dtadj[troot] = prod ? S->dtseed[q] : 0.0;
            for (int t = P->tmpl_count[k] - 1; t >= 0; t--)
                push_adjoint_dev(P, P->tmpl_nodes[k][t], p, S->tval, S->dtval, S->tadj, S->dtadj);
            for (int t = 0; t < P->tmpl_count[k]; t++) {
                const int leafv = P->tmpl_nodes[k][t];
                if (P->nd[leafv].op != O_IDX_VAR) continue;
                int j = i + P->nd[leafv].b;
                if (j < c0 || j >= c1) continue;
                acc_dev(S->dacc, S->ddacc, j - c0, S->tadj[leafv], S->dtadj[leafv], p);
                S->touched[j - c0] = 1;
            }
        }
        const int sv = P->isum_node[k];
        for (int j = c0; j < c1; j++)
            if (S->touched[j - c0]) {
                iv x = iv_mul(S->adj[sv], S->dacc[j - c0], p);
                double dx = dflip(dev_mul(S->adj[sv], S->dadj[sv], S->dacc[j - c0], S->ddacc[j - c0]), x, p);
                acc_dev(S->G, S->dG, j - c0, x, dx, p);
            }
    }
}

/* ------------------------------------------------------------------------ */
/* Exported: problem handle, single-box evaluation, reduction-tree hook      */
/* ------------------------------------------------------------------------ */
void* oracle_create(const void* nodes, int nn, int root, const double* const* tables,
                    const int64_t* tlen, int ntab, int n, const double* l, const double* u,
                    int block) {
    return make_prob(nodes, nn, root, tables, tlen, ntab, n, l, u, block);
}

void oracle_destroy(void* h) { free_prob((oprob*)h); }

int oracle_n_blocks(void* h) { return ((oprob*)h)->nb; }

/* Evaluates one box: F(X) (2 doubles), the midpoint sample F([m, m]) (2),
 * the partials of block blk (2 * B doubles, unused tail left as is) and the
 * monotonicity verdict.  p = 1 evaluates in single precision (the box is
 * widened outward to floats first).  blk < 0 skips the partials. */
int oracle_eval_box(void* h, const double* lo, const double* hi, int p, int blk,
                    double* F, double* Fmid, double* G, int32_t* mono) {
    oprob* P = (oprob*)h;
    obox X = {lo, hi};
    iv f = eval_outer(P, X, p);
    F[0] = f.lo; F[1] = f.hi;
    if (blk >= 0) {
        iv* g = (iv*)malloc(sizeof(iv) * P->B);
        int width = 0;
        block_partials(P, X, p, blk, g, &width);
        for (int t = 0; t < width; t++) { G[2 * t] = g[t].lo; G[2 * t + 1] = g[t].hi; }
        *mono = mono_test(P, X, blk, g, width);
        free(g);
    }
    double* m = (double*)malloc(sizeof(double) * P->n);
    for (int j = 0; j < P->n; j++) m[j] = midpoint(lo[j], hi[j]);
    obox M = {m, m};
    iv fm = eval_outer(P, M, 0);
    Fmid[0] = fm.lo; Fmid[1] = fm.hi;
    free(m);
    return 0;
}

/* oracle_eval_box with the deviation bound of each result: F and its bound
 * dF (1 double, both ends), Fmid and dFmid, the partials of block blk (2 B
 * doubles) and their bounds dG (B doubles).  The values equal
 * oracle_eval_box's. */
int oracle_eval_box_dev(void* h, const double* lo, const double* hi, int p, int blk, double* F, double* dF,
                        double* Fmid, double* dFmid, double* G, double* dG) {
    oprob* P = (oprob*)h;
    dscr S;
    dscr_alloc(P, &S);
    obox X = {lo, hi};
    iv f = dev_outer(P, X, p, &S, dF);
    F[0] = f.lo; F[1] = f.hi;
    if (blk >= 0) {
        int width = 0;
        dev_block_partials(P, X, p, blk, &S, &width);
        for (int t = 0; t < width; t++) {
            G[2 * t] = S.G[t].lo; G[2 * t + 1] = S.G[t].hi;
            dG[t] = S.dG[t];
        }
    }
    double* m = (double*)malloc(sizeof(double) * P->n);
    for (int j = 0; j < P->n; j++) m[j] = midpoint(lo[j], hi[j]);
    obox M = {m, m};
    iv fm = dev_outer(P, M, 0, &S, dFmid);
    Fmid[0] = fm.lo; Fmid[1] = fm.hi;
    free(m);
    dscr_free(&S);
    return 0;
}

/* Test hook: widen every transcendental endpoint by k more ulps (k = 0
 * restores the oracle's rule).  Not thread-safe; used only to perturb the
 * library values when checking the deviation bound. */
void oracle_set_extra_widening(int k) { g_extra_widen = k < 0 ? 0 : k; }

/* Single interval operation, for pinning the arithmetic against an
 * independent multiprecision library.  op uses the node codes; c is the
 * SCALE factor. */
int oracle_iv_op(int op, const double* x, const double* y, double c, int p, double* out) {
    init_constants();
    iv a = mk(x[0], x[1]), b = mk(y[0], y[1]), r;
    switch (op) {
    case O_ADD: r = iv_add(a, b, p); break;
    case O_SUB: r = iv_sub(a, b, p); break;
    case O_MUL: r = iv_mul(a, b, p); break;
    case O_DIV: r = iv_div(a, b, p); break;
    case O_NEG: r = iv_neg(a); break;
    case O_SQR: r = iv_sqr(a, p); break;
    case O_SQRT: r = iv_sqrt(a, p); break;
    case O_EXP: r = iv_exp(a, p); break;
    case O_SIN: r = iv_trig(a, p, 0); break;
    case O_COS: r = iv_trig(a, p, 1); break;
    case O_SCALE: r = iv_scale(a, c, p); break;
    case O_STEP: r = iv_step(a); break;
    case O_PI: r = const_pi(p); break;
    case O_EULER: r = const_e(p); break;
    default: return 1;
    }
    out[0] = r.lo; out[1] = r.hi;
    return 0;
}

/* oracle_iv_op over count operand pairs (x: xlo/xhi, y: ylo/yhi, scale
 * factors c, may be NULL); out: count x 2.  Returns 1 for an unknown op. */
int oracle_iv_op_batch(int op, const double* xlo, const double* xhi, const double* ylo, const double* yhi,
                       const double* c, int64_t count, int p, double* out) {
    for (int64_t k = 0; k < count; k++) {
        const double x[2] = {xlo[k], xhi[k]};
        const double y[2] = {ylo ? ylo[k] : 0.0, yhi ? yhi[k] : 0.0};
        if (oracle_iv_op(op, x, y, c ? c[k] : 0.0, p, out + 2 * k)) return 1;
    }
    return 0;
}

int oracle_tree_prod(const double* lo, const double* hi, int m, int p, double* out) {
    iv* a = (iv*)malloc(sizeof(iv) * (m > 0 ? m : 1));
    for (int i = 0; i < m; i++) a[i] = mk(lo[i], hi[i]);
    iv r = tree_prod(a, m, p);
    out[0] = r.lo; out[1] = r.hi;
    free(a);
    return 0;
}

int oracle_tree_prod_adjoint(const double* lo, const double* hi, int m, double seed_lo, double seed_hi, int p,
                             double* out) {
    iv* a = (iv*)malloc(sizeof(iv) * (m > 0 ? m : 1));
    iv* g = (iv*)malloc(sizeof(iv) * (m > 0 ? m : 1));
    for (int i = 0; i < m; i++) a[i] = mk(lo[i], hi[i]);
    tree_prod_adjoint(a, m, mk(seed_lo, seed_hi), g, p);
    for (int i = 0; i < m; i++) { out[2 * i] = g[i].lo; out[2 * i + 1] = g[i].hi; }
    free(a);
    free(g);
    return 0;
}

int oracle_tree_sum(const double* lo, const double* hi, int m, int p, double* out) {
    iv* a = (iv*)malloc(sizeof(iv) * (m > 0 ? m : 1));
    for (int i = 0; i < m; i++) a[i] = mk(lo[i], hi[i]);
    iv r = tree_sum(a, m, p);
    out[0] = r.lo; out[1] = r.hi;
    free(a);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Branch and bound (section 3.1 flowchart, section 3.2 variable cycling)    */
/* ------------------------------------------------------------------------ */
typedef struct {
    double tol_f, tol_x;
    int32_t split_m, split_d, fp32, samples;   /* samples: 0 midpoint, S > 0 diagonal points */
    int64_t max_gen, max_parents, cap;
    int32_t mono_all;                          /* mono_all: first-order test on every coordinate */
    int32_t threads;                           /* threads for the per-child loops (<= 1: one) */
} oopts;

typedef struct {
    double glb, gub;
    int64_t n_boxes;
    double *box_lo, *box_hi, *box_flo;
    int32_t* box_cyc;
    int64_t generations, evals32, evals64, mids;
    int32_t status, pad;
    int64_t n_trace;
    int64_t *tr_parents, *tr_children, *tr_kept32, *tr_kept, *tr_pool;
    double* tr_gub;
} oresult;

enum { ST_OK = 0, ST_INVALID = 1, ST_CAPACITY = 3, ST_LIMIT = 4 };

typedef struct {
    double *lo, *hi;        /* n each */
    double flo;
    int32_t cyc, fin, blk;  /* cycling position, final flag, block split last */
} entry;

typedef struct { entry* e; int64_t len, cap; } elist;

static void el_push(elist* L, entry x) {
    if (L->len == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 64;
        L->e = (entry*)realloc(L->e, sizeof(entry) * L->cap);
    }
    L->e[L->len++] = x;
}
static void ent_free(entry* x) { free(x->lo); free(x->hi); }

static int cmp_u64(const void* a, const void* b) {
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

static void trace_push(oresult* R, int64_t* cap, int64_t par, int64_t ch, int64_t k32,
                       int64_t k, double gub, int64_t pool) {
    if (R->n_trace == *cap) {
        *cap = *cap ? 2 * *cap : 64;
        R->tr_parents = (int64_t*)realloc(R->tr_parents, sizeof(int64_t) * *cap);
        R->tr_children = (int64_t*)realloc(R->tr_children, sizeof(int64_t) * *cap);
        R->tr_kept32 = (int64_t*)realloc(R->tr_kept32, sizeof(int64_t) * *cap);
        R->tr_kept = (int64_t*)realloc(R->tr_kept, sizeof(int64_t) * *cap);
        R->tr_pool = (int64_t*)realloc(R->tr_pool, sizeof(int64_t) * *cap);
        R->tr_gub = (double*)realloc(R->tr_gub, sizeof(double) * *cap);
    }
    int64_t t = R->n_trace++;
    R->tr_parents[t] = par; R->tr_children[t] = ch; R->tr_kept32[t] = k32;
    R->tr_kept[t] = k; R->tr_gub[t] = gub; R->tr_pool[t] = pool;
}

/* Child r of a box: the d' coordinates starting at the cycling position are
 * each cut into m equal pieces (Eqs. 10-11).  Reading for the rounding of
 * Eqs. 10-11: boundary t of [lo, hi] is RN(lo + RN(RN(RN(hi - lo) / m) * t)),
 * with boundary 0 = lo and boundary m = hi exactly, so the pieces cover the
 * parent.  Digit k of r (base m) picks the piece of coordinate cyc + k. */
static double split_bound(double lo, double hi, int m, int t) {
    if (t == 0) return lo;
    if (t == m) return hi;
    volatile double w = hi - lo;
    volatile double q = w / (double)m;
    volatile double s = q * (double)t;
    volatile double r = lo + s;
    return r;
}

/* GUB samples of a box (section 3.1 lets the sampling be chosen; the paper
 * samples points on the diagonal, section 4).  S = 0: the midpoint; S > 0:
 * the S interior points of the (S + 1)-piece partition of every coordinate
 * taken at the same index j = 1 .. S (the box's diagonal), each coordinate
 * rounded like a split boundary.  Returns the smallest upper end of F at the
 * samples (+inf if none is a number); *count receives the samples taken. */
static double sample_gub(oprob* P, const double* lo, const double* hi, int S, double* pt, int64_t* count) {
    const int n = P->n;
    double best = INFINITY;
    if (S <= 0) {
        for (int j = 0; j < n; j++) pt[j] = midpoint(lo[j], hi[j]);
        obox M = {pt, pt};
        double v = eval_outer(P, M, 0).hi;
        if (v < best) best = v;
        *count += 1;
        return best;
    }
    for (int t = 1; t <= S; t++) {
        for (int j = 0; j < n; j++) pt[j] = split_bound(lo[j], hi[j], S + 1, t);
        obox M = {pt, pt};
        double v = eval_outer(P, M, 0).hi;
        if (v < best) best = v;
    }
    *count += S;
    return best;
}

/* First-order test of the box: on the active block, or (mono_all, the
 * paper's rule of section 3.1) on every coordinate. */
static int mono_box(oprob* P, obox X, int p, int blk, iv* G, int mono_all) {
    int width;
    if (!mono_all) {
        block_partials(P, X, p, blk, G, &width);
        return mono_test(P, X, blk, G, width);
    }
    const int nb = (P->n + P->B - 1) / P->B;
    for (int b = 0; b < nb; b++) {
        block_partials(P, X, p, b, G, &width);
        if (mono_test(P, X, b, G, width)) return 1;
    }
    return 0;
}

/* The per-child passes of a generation: 0 the FP32 test (cut-off against
 * the previous GUB and the first-order test), 1 the GUB samples of the
 * children the FP32 test kept, 2 the FP64 test of those children against
 * the new GUB.  Each job takes the children [q0, q1) with its own copy of
 * the problem's scratch; every result goes to the child's own slot. */
typedef struct {
    oprob* P;
    const oopts* opt;
    entry* kids;
    int64_t q0, q1;
    char *cand, *ok;
    double* fm;
    double gub_prev, gub_new;
    int64_t mids;
    int pass;
    iv* G;
    double* mid;
} cjob;

static void* child_pass(void* arg) {
    cjob* J = (cjob*)arg;
    for (int64_t q = J->q0; q < J->q1; q++) {
        entry* ch = &J->kids[q];
        obox X = {ch->lo, ch->hi};
        if (J->pass == 0) {
            iv f = eval_outer(J->P, X, 1);
            int mono = mono_box(J->P, X, 1, ch->blk, J->G, J->opt->mono_all);
            J->cand[q] = !(f.lo > J->gub_prev) && !mono;
        } else if (J->pass == 1) {
            J->fm[q] = J->cand[q] ? sample_gub(J->P, ch->lo, ch->hi, J->opt->samples, J->mid, &J->mids) : INFINITY;
        } else {
            J->ok[q] = 0;
            if (!J->cand[q]) continue;
            iv f = eval_outer(J->P, X, 0);
            int mono = mono_box(J->P, X, 0, ch->blk, J->G, J->opt->mono_all);
            J->ok[q] = !(f.lo > J->gub_new) && !mono;
            ch->flo = canon_lo(f.lo);
        }
    }
    return NULL;
}

/* Runs pass `pass` over children [0, count) on T jobs (contiguous chunks);
 * job 0 runs on the calling thread. */
static void run_pass(cjob* jobs, int T, int pass, int64_t count) {
    pthread_t tid[256];
    int started[256] = {0};
    for (int t = 0; t < T; t++) {
        jobs[t].pass = pass;
        jobs[t].q0 = count * t / T;
        jobs[t].q1 = count * (t + 1) / T;
    }
    for (int t = 1; t < T; t++)
        started[t] = pthread_create(&tid[t], NULL, child_pass, &jobs[t]) == 0;
    child_pass(&jobs[0]);
    for (int t = 1; t < T; t++) {
        if (started[t]) pthread_join(tid[t], NULL);
        else child_pass(&jobs[t]);   /* no thread: run it here */
    }
}

int oracle_solve(void* h, const oopts* opt, oresult* R) {
    oprob* P = (oprob*)h;
    memset(R, 0, sizeof(*R));
    const int n = P->n, B = P->B, m = opt->split_m, d = opt->split_d, f32 = opt->fp32;
    if (!(m == 2 || m == 4) || d < 1 || d > B || opt->max_parents < 1 || opt->cap < 1 ||
        !(opt->tol_f >= 0.0)) {
        R->status = ST_INVALID;
        return ST_INVALID;
    }
    int64_t tcap = 0;
    iv* G = (iv*)malloc(sizeof(iv) * B);
    double* mid = (double*)malloc(sizeof(double) * n);
    const int T = opt->threads < 1 ? 1 : (opt->threads > 256 ? 256 : opt->threads);
    cjob* jobs = (cjob*)calloc(T, sizeof(cjob));
    for (int t = 0; t < T; t++) {
        jobs[t].P = t == 0 ? P : clone_scratch(P);
        jobs[t].opt = opt;
        jobs[t].G = (iv*)malloc(sizeof(iv) * B);
        jobs[t].mid = (double*)malloc(sizeof(double) * n);
    }

    /* initialisation: the whole domain (section 3.1) */
    elist pool = {0}, par = {0}, kids = {0}, keep = {0};
    entry root;
    root.lo = (double*)malloc(sizeof(double) * n);
    root.hi = (double*)malloc(sizeof(double) * n);
    memcpy(root.lo, P->l, sizeof(double) * n);
    memcpy(root.hi, P->u, sizeof(double) * n);
    obox X0 = {root.lo, root.hi};
    iv f0 = eval_outer(P, X0, 0);
    root.flo = canon_lo(f0.lo);
    root.cyc = 0;
    root.fin = 0;
    R->evals64 = 1;
    double gub = sample_gub(P, root.lo, root.hi, opt->samples, mid, &R->mids);
    if (isnan(gub)) gub = INFINITY;
    el_push(&pool, root);
    int status = ST_OK;
    int64_t gen = 0;

    for (;;) {
        /* remove suboptimal regions: LB > GUB (section 3.1) */
        elist next = {0};
        for (int64_t q = 0; q < pool.len; q++) {
            if (pool.e[q].flo > gub) ent_free(&pool.e[q]);
            else el_push(&next, pool.e[q]);
        }
        free(pool.e); pool = next;
        double thr = d_sub(gub, opt->tol_f, 1);
        int64_t n_act = 0;
        for (int64_t q = 0; q < pool.len; q++)
            if (pool.e[q].flo < thr && !pool.e[q].fin) n_act++;
        if (n_act == 0) break;
        if (gen >= opt->max_gen) { status = ST_LIMIT; break; }

        /* best-first selection, batched: the max_parents active boxes with the
           smallest lower bound; among equal lower bounds at the cut, the ones
           placed last in the list (the most recently inserted) */
        char* sel = (char*)calloc(pool.len, 1);
        if (n_act <= opt->max_parents) {
            for (int64_t q = 0; q < pool.len; q++)
                sel[q] = pool.e[q].flo < thr && !pool.e[q].fin;
        } else {
            uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * n_act);
            int64_t t = 0;
            for (int64_t q = 0; q < pool.len; q++)
                if (pool.e[q].flo < thr && !pool.e[q].fin) keys[t++] = order_key(pool.e[q].flo);
            qsort(keys, n_act, sizeof(uint64_t), cmp_u64);
            uint64_t T = keys[opt->max_parents - 1];
            free(keys);
            int64_t below = 0;
            for (int64_t q = 0; q < pool.len; q++) {
                int act = pool.e[q].flo < thr && !pool.e[q].fin;
                if (act && order_key(pool.e[q].flo) < T) { sel[q] = 1; below++; }
            }
            int64_t need = opt->max_parents - below;
            for (int64_t q = pool.len - 1; q >= 0 && need > 0; q--) {
                int act = pool.e[q].flo < thr && !pool.e[q].fin;
                if (act && order_key(pool.e[q].flo) == T) { sel[q] = 1; need--; }
            }
        }
        par.len = 0;
        next.e = NULL; next.len = next.cap = 0;
        for (int64_t q = 0; q < pool.len; q++) {
            if (sel[q]) el_push(&par, pool.e[q]);
            else el_push(&next, pool.e[q]);
        }
        free(sel);
        free(pool.e); pool = next;

        /* partition each selected region (Eqs. 10-11, variable cycling) */
        kids.len = 0;
        for (int64_t q = 0; q < par.len; q++) {
            const entry* pe = &par.e[q];
            int c = pe->cyc, b = c / B;
            int e = (b + 1) * B < n ? (b + 1) * B : n;
            int dd = d < e - c ? d : e - c;
            int64_t valid = 1;
            for (int k = 0; k < dd; k++) valid *= m;
            for (int64_t r = 0; r < valid; r++) {
                entry ch;
                ch.lo = (double*)malloc(sizeof(double) * n);
                ch.hi = (double*)malloc(sizeof(double) * n);
                memcpy(ch.lo, pe->lo, sizeof(double) * n);
                memcpy(ch.hi, pe->hi, sizeof(double) * n);
                int64_t rr = r;
                for (int k = 0; k < dd; k++) {
                    int dig = (int)(rr % m);
                    rr /= m;
                    int j = c + k;
                    ch.lo[j] = split_bound(pe->lo[j], pe->hi[j], m, dig);
                    ch.hi[j] = split_bound(pe->lo[j], pe->hi[j], m, dig + 1);
                }
                ch.cyc = (c + dd == n) ? 0 : c + dd;
                ch.fin = 0;
                ch.blk = b;
                ch.flo = 0.0;
                el_push(&kids, ch);
            }
        }

        /* sample (GUB update) and rule out (cut-off and first-order test) */
        double gub_prev = gub, gub_new = gub;
        const int64_t nk = kids.len ? kids.len : 1;
        char* cand = (char*)malloc(nk);
        char* okv = (char*)malloc(nk);
        double* fmv = (double*)malloc(sizeof(double) * nk);
        for (int t = 0; t < T; t++) {
            jobs[t].kids = kids.e;
            jobs[t].cand = cand;
            jobs[t].ok = okv;
            jobs[t].fm = fmv;
            jobs[t].gub_prev = gub_prev;
            jobs[t].mids = 0;
        }
        int64_t kept32 = kids.len;
        if (f32) {
            run_pass(jobs, T, 0, kids.len);
            kept32 = 0;
            for (int64_t q = 0; q < kids.len; q++) kept32 += cand[q];
            R->evals32 += kids.len;
        } else {
            memset(cand, 1, kids.len);
        }
        run_pass(jobs, T, 1, kids.len);
        for (int t = 0; t < T; t++) R->mids += jobs[t].mids;
        for (int64_t q = 0; q < kids.len; q++)   /* the minimum is exact: any order gives it */
            if (cand[q] && fmv[q] < gub_new) gub_new = fmv[q];
        for (int t = 0; t < T; t++) jobs[t].gub_new = gub_new;
        run_pass(jobs, T, 2, kids.len);
        keep.len = 0;
        int64_t kept = 0;
        for (int64_t q = 0; q < kids.len; q++) {
            entry* ch = &kids.e[q];
            const int ok = okv[q];
            if (cand[q]) R->evals64++;
            if (ok) {
                int fin = 0;
                if (opt->tol_x > 0.0) {
                    fin = 1;
                    for (int j = 0; j < n; j++)
                        if (!(ch->hi[j] - ch->lo[j] < opt->tol_x)) { fin = 0; break; }
                }
                ch->fin = fin;
                el_push(&keep, *ch);
                kept++;
            } else {
                ent_free(ch);
            }
        }
        free(cand); free(okv); free(fmv);
        /* capacity: boxes alive during the generation.  On overflow the
           generation is abandoned: its children are dropped, its parents go
           back to the end of the list, the samples' GUB is kept, and the
           solve stops with the list still covering every unresolved region. */
        if (pool.len + par.len + keep.len > opt->cap) {
            int64_t npar = par.len;
            for (int64_t q = 0; q < keep.len; q++) ent_free(&keep.e[q]);
            keep.len = 0;
            for (int64_t q = 0; q < par.len; q++) el_push(&pool, par.e[q]);
            par.len = 0;
            gub = gub_new;
            status = ST_CAPACITY;
            gen++;
            trace_push(R, &tcap, npar, kids.len, kept32, 0, gub, pool.len);
            break;
        }
        for (int64_t q = 0; q < par.len; q++) ent_free(&par.e[q]);
        for (int64_t q = 0; q < keep.len; q++) el_push(&pool, keep.e[q]);
        gub = gub_new;
        gen++;
        trace_push(R, &tcap, par.len, kids.len, kept32, kept, gub, pool.len);
    }

    /* output (section 3.1): regions with LB <= GUB, GLB = their smallest LB */
    elist out = {0};
    for (int64_t q = 0; q < pool.len; q++) {
        if (pool.e[q].flo > gub) ent_free(&pool.e[q]);
        else el_push(&out, pool.e[q]);
    }
    free(pool.e);
    double glb = INFINITY;
    for (int64_t q = 0; q < out.len; q++) if (out.e[q].flo < glb) glb = out.e[q].flo;
    R->glb = glb;
    R->gub = gub;
    R->n_boxes = out.len;
    R->box_lo = (double*)malloc(sizeof(double) * n * (out.len ? out.len : 1));
    R->box_hi = (double*)malloc(sizeof(double) * n * (out.len ? out.len : 1));
    R->box_flo = (double*)malloc(sizeof(double) * (out.len ? out.len : 1));
    R->box_cyc = (int32_t*)malloc(sizeof(int32_t) * (out.len ? out.len : 1));
    for (int64_t q = 0; q < out.len; q++) {
        memcpy(R->box_lo + q * n, out.e[q].lo, sizeof(double) * n);
        memcpy(R->box_hi + q * n, out.e[q].hi, sizeof(double) * n);
        R->box_flo[q] = out.e[q].flo;
        R->box_cyc[q] = out.e[q].cyc;
        ent_free(&out.e[q]);
    }
    free(out.e); free(par.e); free(kids.e); free(keep.e);
    free(G); free(mid);
    for (int t = 0; t < T; t++) {
        free(jobs[t].G);
        free(jobs[t].mid);
        if (t > 0) free_clone(jobs[t].P);
    }
    free(jobs);
    R->generations = gen;
    R->status = status;
    return status;
}

void oracle_free_result(oresult* R) {
    free(R->box_lo); free(R->box_hi); free(R->box_flo); free(R->box_cyc);
    free(R->tr_parents); free(R->tr_children); free(R->tr_kept32); free(R->tr_kept);
    free(R->tr_pool); free(R->tr_gub);
    memset(R, 0, sizeof(*R));
}
