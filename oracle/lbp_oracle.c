/*
 * FP64 CPU oracle for log-space loopy belief propagation over a flat factor graph.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library; the product path never does. It shares no
 * code, header, table or constant with the CUDA path.
 *
 * What it computes (PGMax, arXiv 2202.04110):
 *   - LBP on discrete factor graphs (Sec. 1, Pearl 1988 / Murphy 1999), in log space,
 *     with parallel ("flooding") message updates and damping (Sec. 3, Pretti 2005):
 *     every new factor-to-variable message of iteration t is computed from the
 *     messages of iteration t-1.
 *   - Enumeration factors given by their list of valid configurations and one
 *     log-potential per configuration (Sec. 5.2). Unlisted configurations have
 *     potential -inf.
 *   - Logical OR / AND / XOR factors with message updates linear in the fan-in (Sec. 3;
 *     the paper counts three kinds and names none; XOR, the parity check, is the third
 *     taken here).
 *   - Temperature T on the factor log-sum-exp: T = 1 is sum-product, T = 0 is the
 *     max-product limit used for MAP (Sec. 5.1).
 *   - MAP decode: per-variable argmax of the beliefs (Sec. 5.1), lowest state on ties.
 *
 * Steps of one iteration, in this order:
 *   (i)   variable to factor: m_{v->f}(x) = e_v(x) + sum_{g in N(v), g != f} m_{g->v}(x),
 *         as an explicit leave-one-out sum (prefix + suffix), never a subtraction;
 *   (ii)  factor to variable, enumeration:
 *           mt_{f->i}(x) = LSE_T over c in C_f with c_i = x of
 *                          [ phi_f(c) + sum_{j != i} m_{j->f}(c_j) ]
 *         logical: the closed forms in or_update() (brute force in or_update_brute());
 *   (iii) mt is max-normalised (its additive constant is free), then damped,
 *           m_t = delta * m_{t-1} + (1 - delta) * mt      (m_t = mt when delta = 0),
 *         then max-normalised again. An all -inf message is a contradiction: it is
 *         replaced by zeros and flag bit 0 is raised.
 * Beliefs after the last iteration: b_v = e_v + sum_f m_{f->v}; normalised log-beliefs
 * b_v - LSE_1(b_v).
 *
 * Flat layouts (shared interface definition with the CUDA path, restated here):
 *   evidence/beliefs variable-major; messages edge-major with edges enumerated group by
 *   group (enumeration groups, then logical groups), factor-major, an enumeration
 *   factor's neighbours in order, a logical factor's parents then its child.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OG_OR 0
#define OG_AND 1
#define OG_XOR 2
#define OG_FLAG_CONTRADICTION 1u
#define OG_FLAG_NAN 2u
#define PGM_ORACLE_KMAX 256

typedef struct {
    int32_t n_vars;
    const int32_t *num_states;
    int32_t n_enum;
    const int32_t *e_arity, *e_ncfg, *e_nfac, *e_shared;
    const int32_t *const *e_cfg;  /* per group [n_cfg * arity] */
    const int32_t *const *e_vars; /* per group [n_fac * arity] */
    int32_t n_logic;
    const int32_t *l_kind, *l_nfac;
    const int32_t *const *l_paroff;  /* per group [n_fac + 1] */
    const int32_t *const *l_parents; /* per group [par_off[n_fac]] */
    const int32_t *const *l_child;   /* per group [n_fac] */
} og_graph;

/* ---- scalar helpers ------------------------------------------------------------ */

static double lse_T(const double *z, int n, double T) {
    /* LSE_T(z) = T log sum exp(z/T) for T > 0; max(z) for T = 0. Empty set: -inf. */
    double m = -INFINITY;
    for (int k = 0; k < n; ++k)
        if (z[k] > m) m = z[k];
    if (T == 0.0 || m == -INFINITY || m == INFINITY) return m;
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += exp((z[k] - m) / T);
    return m + T * log(s);
}

static void normalise(double *m, int K, uint32_t *flags) {
    double mx = -INFINITY;
    int has_nan = 0;
    for (int x = 0; x < K; ++x) {
        if (isnan(m[x])) has_nan = 1;
        else if (m[x] > mx) mx = m[x];
    }
    if (has_nan) *flags |= OG_FLAG_NAN;
    if (mx == -INFINITY) {
        for (int x = 0; x < K; ++x) m[x] = 0.0;
        *flags |= OG_FLAG_CONTRADICTION;
        return;
    }
    for (int x = 0; x < K; ++x) m[x] -= mx;
}

/* ---- logical factors ------------------------------------------------------------ */

/*
 * OR factor, child c = OR(p_1..p_n), binary variables, potential 0 on valid
 * configurations. Inputs are the incoming log-odds x_j = m_{p_j->f}(1) - m_{p_j->f}(0)
 * and x_c for the child. Outputs are the outgoing log-odds out[0..n-1] to the parents
 * and out[n] to the child. Derivation (sum over parent configurations, T > 0):
 *   A = sum_j sp_T(x_j),  A_{-i} = sum_{j != i} sp_T(x_j),
 *   to child:  L_T(A)                                   (all-zero parents excluded)
 *   to parent: x_c + A_{-i} - sp_T(x_c + L_T(A_{-i}))
 * and the T = 0 limit with S_{-i} = sum_{j != i} max(x_j, 0), M_{-i} = max_{j != i} x_j:
 *   to child:  sum_j max(x_j, 0) + min(0, max_j x_j)
 *   to parent: x_c + S_{-i} - max(0, x_c + S_{-i} + min(0, M_{-i})).
 * The parent formulas are evaluated in an algebraically equal form that stays finite
 * when x_c or A_{-i} is infinite. Leave-one-out sums are prefix + suffix, O(n).
 * For T > 0 the sums A are accumulated as logarithms (log A = LSE_j log sp_T(x_j)), so
 * that very negative log-odds, whose softplus underflows, still give log A ~ x_j.
 */

/* log(s(u)) with s(u) = log(1 + e^u): for u < -30, s(u) = e^u (1 - e^u/2 + ...);
 * for u > 0, s(u) = u + log(1 + e^-u). */
static double log_softplus(double u) {
    if (u < -30.0) return u + log1p(-0.5 * exp(u));
    if (u > 0.0) return log(u + log1p(exp(-u)));
    return log(log1p(exp(u)));
}

static double lse2(double a, double b) {
    double m = a > b ? a : b;
    if (m == -INFINITY || m == INFINITY) return m;
    return m + log(exp(a - m) + exp(b - m));
}

/* L(s) = log(e^s - 1) from ls = log s (s = sum of softplus terms, dimensionless). */
static double log_expm1_from_log(double ls) {
    if (ls == -INFINITY) return -INFINITY;
    if (ls == INFINITY) return INFINITY;
    if (ls > 0.0) {
        double s = exp(ls);
        return s + log(-expm1(-s));
    }
    if (ls > -700.0) {
        double s = exp(ls);
        return ls + log(expm1(s) / s);
    }
    return ls;
}

/* -log(1 - e^{-s}) from ls = log s. */
static double neg_log_1mexp_from_log(double ls) {
    if (ls == INFINITY) return 0.0;
    if (ls > 0.0) return -log(-expm1(-exp(ls)));
    if (ls > -700.0) {
        double s = exp(ls);
        return -ls - log(-expm1(-s) / s);
    }
    return -ls;
}

static void or_update(int n, const double *x, double xc, double T, double *out) {
    double *pre = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    double *suf = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    double *pmax = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    double *smax = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    if (T == 0.0) {
        pre[0] = 0.0;
        pmax[0] = -INFINITY;
        for (int j = 0; j < n; ++j) {
            pre[j + 1] = pre[j] + (x[j] > 0.0 ? x[j] : 0.0);
            pmax[j + 1] = x[j] > pmax[j] ? x[j] : pmax[j];
        }
        suf[n] = 0.0;
        smax[n] = -INFINITY;
        for (int j = n - 1; j >= 0; --j) {
            suf[j] = suf[j + 1] + (x[j] > 0.0 ? x[j] : 0.0);
            smax[j] = x[j] > smax[j + 1] ? x[j] : smax[j + 1];
        }
        double mall = pmax[n];
        out[n] = pre[n] + (mall < 0.0 ? mall : 0.0);
        for (int i = 0; i < n; ++i) {
            double S = pre[i] + suf[i + 1];
            double M = pmax[i] > smax[i + 1] ? pmax[i] : smax[i + 1];
            double mn = M < 0.0 ? M : 0.0;
            double z = xc + S + mn;
            out[i] = (z >= 0.0) ? -mn : xc + S;
        }
    } else {
        /* pre/suf hold log of the (dimensionless) softplus sums sum s(x_j / T) */
        pre[0] = -INFINITY;
        for (int j = 0; j < n; ++j) pre[j + 1] = lse2(pre[j], log_softplus(x[j] / T));
        suf[n] = -INFINITY;
        for (int j = n - 1; j >= 0; --j) suf[j] = lse2(suf[j + 1], log_softplus(x[j] / T));
        out[n] = T * log_expm1_from_log(pre[n]);
        for (int i = 0; i < n; ++i) {
            double ls = lse2(pre[i], suf[i + 1]);
            if (ls == -INFINITY) {
                out[i] = xc;
                continue;
            }
            double y = xc + T * log_expm1_from_log(ls);
            if (y >= 0.0)
                out[i] = T * neg_log_1mexp_from_log(ls) - T * log1p(exp(-y / T));
            else
                out[i] = xc + T * exp(ls) - T * log1p(exp(y / T));
        }
    }
    free(pre);
    free(suf);
    free(pmax);
    free(smax);
}

/* The child's value for parent configuration p: OR, AND, or XOR (the parity of the
 * parents; the factor admits exactly the configurations of even total parity). */
static int logic_child(int kind, int any, int all, int64_t p, int n) {
    if (kind == OG_OR) return any;
    if (kind == OG_AND) return all;
    int par = 0;
    for (int j = 0; j < n; ++j) par ^= (int)((p >> j) & 1);
    return par;
}

/*
 * Brute force over all 2^n parent configurations (the definition the closed form must
 * reproduce). v2f holds the incoming 2-vectors, parents then child. mt receives the
 * outgoing raw (unnormalised) 2-vectors in the same order.
 */
static void logic_brute(int kind, int n, const double *v2f, double T, double *mt) {
    int ne = n + 1;
    int64_t nconf = (int64_t)1 << n;
    double *vals = (double *)malloc(sizeof(double) * (size_t)nconf);
    for (int i = 0; i < ne; ++i) {
        for (int xi = 0; xi < 2; ++xi) {
            int cnt = 0;
            for (int64_t p = 0; p < nconf; ++p) {
                int any = 0, all = 1;
                for (int j = 0; j < n; ++j) {
                    int bit = (int)((p >> j) & 1);
                    any |= bit;
                    all &= bit;
                }
                int c = logic_child(kind, any, all, p, n);
                int state_i = (i < n) ? (int)((p >> i) & 1) : c;
                if (state_i != xi) continue;
                double s = 0.0;
                for (int j = 0; j < n; ++j)
                    if (j != i) s += v2f[2 * j + ((p >> j) & 1)];
                if (i != n) s += v2f[2 * n + c];
                vals[cnt++] = s;
            }
            mt[2 * i + xi] = lse_T(vals, cnt, T);
        }
    }
    free(vals);
}

static double log_odds(const double *m2) {
    if (m2[0] == -INFINITY && m2[1] == -INFINITY) return 0.0;
    return m2[1] - m2[0];
}

/*
 * XOR factor, child c = XOR(p_1..p_n): the n + 1 variables have even total parity, so
 * every member's message depends on all the others alike. With log-odds a_j = x_j / T of
 * the others, summing their configurations of each parity gives (the product rule of
 * parity checks)
 *   D = prod_{j != i} tanh(-a_j / 2),   out_i = T log((1 - D) / (1 + D)),
 * and the T = 0 limit (max over configurations: flip the cheapest of the others when the
 * best configuration has the wrong parity)
 *   out_i = -(prod_{j != i} s_j) min_{j != i} |x_j|,   s_j = -1 if x_j > 0 else +1.
 * An empty set of others (the child of a parentless factor) gives D = 1, out = -inf.
 * For T > 0 the product is kept as a sign and the magnitude as
 *   u_j = -log |tanh(a_j / 2)| >= 0,  held as l_j = log u_j,
 * so that log |D| = -sum_j u_j keeps its precision when every other member is decided
 * (u_j ~ 2 e^{-|a_j|}, far below the smallest double): lambda = LSE_{j != i} l_j and
 *   log((1 - |D|) / (1 + |D|)) = log(-expm1(-e^lambda)) - log1p(e^{-e^lambda}),
 * which is lambda - log 2 to double precision once e^lambda < 1e-9. Leave-one-out values
 * are prefix + suffix, O(n). x holds the n + 1 members' log-odds.
 */
/* log u with u = -log tanh(|a| / 2) = log1p(2 / expm1(|a|)); for |a| > 30,
 * u = 2 e^{-|a|} (1 + O(e^{-|a|})), so log u = log 2 - |a| to 1e-13. */
static double log_u_tanh_half(double a) {
    a = fabs(a);
    if (a == 0.0) return INFINITY;       /* tanh 0 = 0: u = +inf */
    if (a == INFINITY) return -INFINITY; /* tanh = 1: u = 0 */
    if (a > 30.0) return log(2.0) - a;
    return log(log1p(2.0 / expm1(a)));
}

static void xor_update(int m, const double *x, double T, double *out) {
    double *pl = (double *)malloc(sizeof(double) * (size_t)(m + 1));
    double *sl = (double *)malloc(sizeof(double) * (size_t)(m + 1));
    int *ps = (int *)malloc(sizeof(int) * (size_t)(m + 1));
    int *ss = (int *)malloc(sizeof(int) * (size_t)(m + 1));
    if (T == 0.0) {
        /* pl / sl: prefix / suffix minima of |x|; ps / ss: parities of the positive x */
        pl[0] = INFINITY;
        ps[0] = 0;
        for (int j = 0; j < m; ++j) {
            pl[j + 1] = fabs(x[j]) < pl[j] ? fabs(x[j]) : pl[j];
            ps[j + 1] = ps[j] ^ (x[j] > 0.0);
        }
        sl[m] = INFINITY;
        ss[m] = 0;
        for (int j = m - 1; j >= 0; --j) {
            sl[j] = fabs(x[j]) < sl[j + 1] ? fabs(x[j]) : sl[j + 1];
            ss[j] = ss[j + 1] ^ (x[j] > 0.0);
        }
        for (int i = 0; i < m; ++i) {
            double mn = pl[i] < sl[i + 1] ? pl[i] : sl[i + 1];
            int odd = ps[i] ^ ss[i + 1];
            out[i] = odd ? mn : -mn;
        }
    } else {
        /* pl / sl: prefix / suffix LSE of l_j; ps / ss: parities of the positive x (the
         * negative factors tanh(-a_j / 2)) */
        pl[0] = -INFINITY;
        ps[0] = 0;
        for (int j = 0; j < m; ++j) {
            pl[j + 1] = lse2(pl[j], log_u_tanh_half(x[j] / T));
            ps[j + 1] = ps[j] ^ (x[j] > 0.0);
        }
        sl[m] = -INFINITY;
        ss[m] = 0;
        for (int j = m - 1; j >= 0; --j) {
            sl[j] = lse2(sl[j + 1], log_u_tanh_half(x[j] / T));
            ss[j] = ss[j + 1] ^ (x[j] > 0.0);
        }
        for (int i = 0; i < m; ++i) {
            double lam = lse2(pl[i], sl[i + 1]);
            int neg = ps[i] ^ ss[i + 1]; /* D < 0 */
            double r;                    /* log((1 - |D|) / (1 + |D|)) <= 0 */
            if (lam == INFINITY) r = 0.0;
            else if (lam == -INFINITY) r = -INFINITY;
            else if (lam < -20.7) r = lam - log(2.0);
            else {
                double u = exp(lam);
                r = log(-expm1(-u)) - log1p(exp(-u));
            }
            out[i] = T * (neg ? -r : r);
        }
    }
    free(pl);
    free(sl);
    free(ps);
    free(ss);
}

/* Closed-form logical update; v2f and mt as in logic_brute(); mt is normalised. */
static void logic_closed(int kind, int n, const double *v2f, double T, double *mt) {
    if (kind == OG_XOR) {
        double *x = (double *)malloc(sizeof(double) * (size_t)(n + 1));
        double *out = (double *)malloc(sizeof(double) * (size_t)(n + 1));
        for (int j = 0; j <= n; ++j) x[j] = log_odds(v2f + 2 * j);
        xor_update(n + 1, x, T, out);
        for (int i = 0; i <= n; ++i) {
            double o = out[i];
            if (o >= 0.0) {
                mt[2 * i] = -o;
                mt[2 * i + 1] = 0.0;
            } else {
                mt[2 * i] = 0.0;
                mt[2 * i + 1] = o;
            }
        }
        free(x);
        free(out);
        return;
    }
    double sgn = (kind == OG_AND) ? -1.0 : 1.0; /* AND(p) = not OR(not p) */
    double *x = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    double *out = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    for (int j = 0; j < n; ++j) x[j] = sgn * log_odds(v2f + 2 * j);
    double xc = sgn * log_odds(v2f + 2 * n);
    or_update(n, x, xc, T, out);
    for (int i = 0; i <= n; ++i) {
        double o = sgn * out[i];
        if (o >= 0.0) {
            mt[2 * i] = -o;
            mt[2 * i + 1] = 0.0;
        } else {
            mt[2 * i] = 0.0;
            mt[2 * i + 1] = o;
        }
    }
    free(x);
    free(out);
}

/* ---- graph layout ----------------------------------------------------------------- */

typedef struct {
    int64_t V, VS, E, ES;
    int64_t *vs_off;   /* [V+1] */
    int32_t *edge_var; /* [E] */
    int64_t *es_off;   /* [E+1] */
    int64_t *vin_off;  /* [V+1] CSR of incoming edges per variable */
    int64_t *vin_edge; /* [E] edge ids, ascending */
    int64_t *enum_edge0, *logic_edge0; /* first edge of each group */
    int64_t *enum_pot0;                /* first log-potential of each group */
} og_layout;

static void layout_free(og_layout *L) {
    free(L->vs_off);
    free(L->edge_var);
    free(L->es_off);
    free(L->vin_off);
    free(L->vin_edge);
    free(L->enum_edge0);
    free(L->logic_edge0);
    free(L->enum_pot0);
}

static void layout_build(const og_graph *g, og_layout *L) {
    L->V = g->n_vars;
    L->vs_off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(L->V + 1));
    L->vs_off[0] = 0;
    for (int64_t v = 0; v < L->V; ++v) L->vs_off[v + 1] = L->vs_off[v] + g->num_states[v];
    L->VS = L->vs_off[L->V];
    int64_t E = 0;
    for (int k = 0; k < g->n_enum; ++k) E += (int64_t)g->e_nfac[k] * g->e_arity[k];
    for (int k = 0; k < g->n_logic; ++k) E += (int64_t)g->l_paroff[k][g->l_nfac[k]] + g->l_nfac[k];
    L->E = E;
    L->edge_var = (int32_t *)malloc(sizeof(int32_t) * (size_t)(E > 0 ? E : 1));
    L->enum_edge0 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(g->n_enum + 1));
    L->logic_edge0 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(g->n_logic + 1));
    L->enum_pot0 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(g->n_enum + 1));
    int64_t e = 0, p = 0;
    for (int k = 0; k < g->n_enum; ++k) {
        L->enum_edge0[k] = e;
        L->enum_pot0[k] = p;
        int64_t n = (int64_t)g->e_nfac[k] * g->e_arity[k];
        for (int64_t i = 0; i < n; ++i) L->edge_var[e++] = g->e_vars[k][i];
        p += g->e_shared[k] ? g->e_ncfg[k] : (int64_t)g->e_ncfg[k] * g->e_nfac[k];
    }
    for (int k = 0; k < g->n_logic; ++k) {
        L->logic_edge0[k] = e;
        for (int f = 0; f < g->l_nfac[k]; ++f) {
            for (int32_t q = g->l_paroff[k][f]; q < g->l_paroff[k][f + 1]; ++q)
                L->edge_var[e++] = g->l_parents[k][q];
            L->edge_var[e++] = g->l_child[k][f];
        }
    }
    L->es_off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(E + 1));
    L->es_off[0] = 0;
    for (int64_t i = 0; i < E; ++i) L->es_off[i + 1] = L->es_off[i] + g->num_states[L->edge_var[i]];
    L->ES = L->es_off[E];
    L->vin_off = (int64_t *)calloc((size_t)(L->V + 1), sizeof(int64_t));
    for (int64_t i = 0; i < E; ++i) L->vin_off[L->edge_var[i] + 1]++;
    for (int64_t v = 0; v < L->V; ++v) L->vin_off[v + 1] += L->vin_off[v];
    L->vin_edge = (int64_t *)malloc(sizeof(int64_t) * (size_t)(E > 0 ? E : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(L->V + 1));
    memcpy(fill, L->vin_off, sizeof(int64_t) * (size_t)(L->V + 1));
    for (int64_t i = 0; i < E; ++i) L->vin_edge[fill[L->edge_var[i]]++] = i;
    free(fill);
}

/* (i) variable-to-factor messages by explicit leave-one-out (prefix + suffix) */
static void var_to_factor(const og_graph *g, const og_layout *L, const double *evidence,
                          const double *msgs, double *v2f) {
    (void)g;
#pragma omp parallel
    {
        int64_t cap = 16;
        double *pre = (double *)malloc(sizeof(double) * (size_t)cap);
#pragma omp for schedule(dynamic, 64)
        for (int64_t v = 0; v < L->V; ++v) {
            int64_t d = L->vin_off[v + 1] - L->vin_off[v];
            if (d + 1 > cap) {
                cap = d + 1;
                pre = (double *)realloc(pre, sizeof(double) * (size_t)cap);
            }
            int K = (int)(L->vs_off[v + 1] - L->vs_off[v]);
            for (int x = 0; x < K; ++x) {
                pre[0] = evidence[L->vs_off[v] + x];
                for (int64_t k = 0; k < d; ++k) {
                    int64_t ed = L->vin_edge[L->vin_off[v] + k];
                    pre[k + 1] = pre[k] + msgs[L->es_off[ed] + x];
                }
                double suf = 0.0;
                for (int64_t k = d - 1; k >= 0; --k) {
                    int64_t ed = L->vin_edge[L->vin_off[v] + k];
                    v2f[L->es_off[ed] + x] = pre[k] + suf;
                    suf += msgs[L->es_off[ed] + x];
                }
            }
        }
        free(pre);
    }
}

/* (ii) enumeration factor to variable, raw (unnormalised) */
static void enum_factor(const og_graph *g, const og_layout *L, int k, int64_t f,
                        const double *log_pot, double T, const double *v2f, double *mt,
                        double *vals) {
    int a = g->e_arity[k], nc = g->e_ncfg[k];
    const int32_t *cfg = g->e_cfg[k];
    int64_t e0 = L->enum_edge0[k] + f * a;
    const double *phi = log_pot + L->enum_pot0[k] + (g->e_shared[k] ? 0 : f * nc);
    for (int i = 0; i < a; ++i) {
        int Ki = g->num_states[L->edge_var[e0 + i]];
        for (int x = 0; x < Ki; ++x) {
            int cnt = 0;
            for (int c = 0; c < nc; ++c) {
                if (cfg[c * a + i] != x) continue;
                double s = phi[c];
                for (int j = 0; j < a; ++j)
                    if (j != i) s += v2f[L->es_off[e0 + j] + cfg[c * a + j]];
                vals[cnt++] = s;
            }
            mt[L->es_off[e0 + i] + x] = lse_T(vals, cnt, T);
        }
    }
}

static void damp_normalise(double *mnew, const double *mold, int K, double damping,
                           uint32_t *flags) {
    normalise(mnew, K, flags);
    if (damping != 0.0)
        for (int x = 0; x < K; ++x) mnew[x] = damping * mold[x] + (1.0 - damping) * mnew[x];
    normalise(mnew, K, flags);
}

static int64_t max_ncfg(const og_graph *g) {
    int64_t m = 2;
    for (int k = 0; k < g->n_enum; ++k)
        if (g->e_ncfg[k] > m) m = g->e_ncfg[k];
    return m;
}

int og_sizes(const og_graph *g, int64_t *out6) {
    og_layout L;
    layout_build(g, &L);
    int64_t P = 0;
    for (int k = 0; k < g->n_enum; ++k)
        P += g->e_shared[k] ? g->e_ncfg[k] : (int64_t)g->e_ncfg[k] * g->e_nfac[k];
    out6[0] = L.V;
    out6[1] = L.VS;
    out6[2] = L.E;
    out6[3] = L.ES;
    out6[4] = P;
    out6[5] = 0;
    layout_free(&L);
    return 0;
}

/*
 * n_iters flooding iterations starting from the messages in msgs ([ES], in/out; zeros
 * for a cold start). use_brute = 1 evaluates logical factors by brute force.
 * round_f32 = 1 rounds the messages to FP32 after every iteration (the arithmetic stays
 * FP64): a model of FP32 message storage, used to measure how far FP32 storage alone
 * moves a run.
 */
int og_bp(const og_graph *g, const double *log_pot, const double *evidence, double T,
          double damping, int n_iters, int use_brute, int round_f32, double *msgs,
          uint32_t *flags) {
    if (T < 0.0 || damping < 0.0 || damping >= 1.0 || n_iters < 0) return -1;
    og_layout L;
    layout_build(g, &L);
    size_t ES = (size_t)(L.ES > 0 ? L.ES : 1);
    double *v2f = (double *)malloc(sizeof(double) * ES);
    double *mt = (double *)malloc(sizeof(double) * ES);
    int64_t ncmax = max_ncfg(g);
    uint32_t fl = 0;
    for (int it = 0; it < n_iters; ++it) {
        var_to_factor(g, &L, evidence, msgs, v2f);
        for (int k = 0; k < g->n_enum; ++k) {
#pragma omp parallel
            {
                double *vals = (double *)malloc(sizeof(double) * (size_t)ncmax);
#pragma omp for schedule(static)
                for (int64_t f = 0; f < g->e_nfac[k]; ++f)
                    enum_factor(g, &L, k, f, log_pot, T, v2f, mt, vals);
                free(vals);
            }
        }
        for (int k = 0; k < g->n_logic; ++k) {
            const int32_t *po = g->l_paroff[k];
#pragma omp parallel for schedule(dynamic, 64)
            for (int64_t f = 0; f < g->l_nfac[k]; ++f) {
                int n = po[f + 1] - po[f];
                int64_t e0 = L.logic_edge0[k] + po[f] + f; /* one child edge per earlier factor */
                int64_t s0 = L.es_off[e0];
                if (use_brute)
                    logic_brute(g->l_kind[k], n, v2f + s0, T, mt + s0);
                else
                    logic_closed(g->l_kind[k], n, v2f + s0, T, mt + s0);
            }
        }
        uint32_t itfl = 0;
#pragma omp parallel for schedule(static) reduction(| : itfl)
        for (int64_t e = 0; e < L.E; ++e) {
            int K = (int)(L.es_off[e + 1] - L.es_off[e]);
            damp_normalise(mt + L.es_off[e], msgs + L.es_off[e], K, damping, &itfl);
        }
        fl |= itfl;
        memcpy(msgs, mt, sizeof(double) * (size_t)L.ES);
        /* storage model of an implementation that keeps its messages in FP32 */
        if (round_f32)
            for (int64_t i = 0; i < L.ES; ++i) msgs[i] = (double)(float)msgs[i];
    }
    if (flags) *flags |= fl;
    free(v2f);
    free(mt);
    layout_free(&L);
    return 0;
}

/*
 * Beliefs b_v = e_v + sum_f m_{f->v}. Writes the unnormalised beliefs (if raw != NULL),
 * the normalised log-beliefs b - LSE_1(b) (if normed != NULL) and the argmax decode,
 * lowest state on ties (if decode != NULL). A variable whose beliefs are all -inf is a
 * contradiction: normalised beliefs stay -inf, decode is 0, flag bit 0 is raised.
 */
int og_beliefs(const og_graph *g, const double *evidence, const double *msgs, double *raw,
               double *normed, int32_t *decode, uint32_t *flags) {
    og_layout L;
    layout_build(g, &L);
    uint32_t fl = 0;
    int32_t kmax = 1;
    for (int64_t v = 0; v < L.V; ++v)
        if (g->num_states[v] > kmax) kmax = g->num_states[v];
#pragma omp parallel reduction(| : fl)
    {
        double *b = (double *)malloc(sizeof(double) * (size_t)kmax);
#pragma omp for schedule(dynamic, 64)
        for (int64_t v = 0; v < L.V; ++v) {
            int K = g->num_states[v];
            for (int x = 0; x < K; ++x) {
                double s = evidence[L.vs_off[v] + x];
                for (int64_t q = L.vin_off[v]; q < L.vin_off[v + 1]; ++q)
                    s += msgs[L.es_off[L.vin_edge[q]] + x];
                b[x] = s;
            }
            int arg = 0;
            for (int x = 1; x < K; ++x)
                if (b[x] > b[arg]) arg = x;
            double z = lse_T(b, K, 1.0);
            if (z == -INFINITY) fl |= OG_FLAG_CONTRADICTION;
            for (int x = 0; x < K; ++x) {
                if (isnan(b[x])) fl |= OG_FLAG_NAN;
                if (raw) raw[L.vs_off[v] + x] = b[x];
                if (normed) normed[L.vs_off[v] + x] = (z == -INFINITY) ? -INFINITY : b[x] - z;
            }
            if (decode) decode[v] = arg;
        }
        free(b);
    }
    if (flags) *flags |= fl;
    layout_free(&L);
    return 0;
}

/*
 * One logical factor in isolation: v2f = incoming 2-vectors (parents, then child);
 * mt = outgoing normalised 2-vectors. brute = 1 uses the enumeration definition.
 */
int og_logic_update(int kind, int n, const double *v2f, double T, int brute, double *mt) {
    if (brute) {
        logic_brute(kind, n, v2f, T, mt);
        uint32_t fl = 0;
        for (int i = 0; i <= n; ++i) normalise(mt + 2 * i, 2, &fl);
    } else {
        logic_closed(kind, n, v2f, T, mt);
    }
    return 0;
}

int og_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the following calls (n >= 1; timing only: every result is independent of
 * the thread count, each factor and variable being computed by one thread). Returns the
 * count in effect. */
int og_set_num_threads(int n) {
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ---- adjoint (gradient) -------------------------------------------------------------- */

/* argmax over K values, lowest index on ties */
static int argmax_k(const double *m, int K) {
    int a = 0;
    for (int x = 1; x < K; ++x)
        if (m[x] > m[a]) a = x;
    return a;
}

/*
 * Gradient of L = sum_v sum_x g[v,x] * nb[v,x], nb = b - LSE_1(b), the normalised
 * log-beliefs after n_iters flooding iterations from zero messages, with respect to the
 * log-potentials and the evidence (the "grad" of Sec. 5.3: LBP inside a differentiable
 * system). T > 0; logical factors of fan-in at most 20 (returns -2 for larger ones).
 * Reverse-mode chain rule through each forward step, in reverse order:
 *   beliefs   nb = b - LSE(b):         db = g - softmax(b) * sum(g)
 *   b = e + sum m:                     de += db, dm_{g->v} += db
 *   normalise m_t = d - d[argmax]:     dd = dm - (sum dm) * onehot(argmax)
 *   damping d = delta m_{t-1} + (1 - delta) n:   dm_{t-1} += delta dd, dn = (1 - delta) dd
 *   normalise n = mt - mt[argmax]:     dmt = dn - (sum dn) * onehot(argmax)
 *   factor mt_i(x) = T log sum_{c: c_i = x} exp(s_{-i}(c) / T), s_{-i}(c) = phi(c) + sum_{j != i} v_j(c_j):
 *       with p = exp((s_{-i}(c) - mt_i(c_i)) / T):  dphi(c) += dmt_i(c_i) p,  dv_j(c_j) += dmt_i(c_i) p (j != i)
 *   logical factor: the same softmax rule over its valid configurations (parents' states
 *       p, child c = OR(p) or AND(p), log-potential 0), the outgoing 2-vectors taken as
 *       their enumerated LSE values (logic_brute; the closed form's normalised output
 *       differs from them by a constant per edge, which the normalisation removes)
 *   leave-one-out v_{f->v} = e_v + sum_{g != f} m_{g->v}:  de += dv,  dm_{g->v} += dv (g != f)
 * All intermediate message states are kept (small graphs).
 */
int og_grad(const og_graph *g, const double *log_pot, const double *evidence, double T, double damping,
            int n_iters, const double *g_nb, double *d_log_pot, double *d_evidence) {
    if (!(T > 0.0) || damping < 0.0 || damping >= 1.0 || n_iters < 0) return -1;
    for (int k = 0; k < g->n_logic; ++k)
        for (int64_t f = 0; f < g->l_nfac[k]; ++f)
            if (g->l_paroff[k][f + 1] - g->l_paroff[k][f] > 20) return -2;
    og_layout L;
    layout_build(g, &L);
    const int64_t ES = L.ES, VS = L.VS;
    int64_t P = 0;
    for (int k = 0; k < g->n_enum; ++k) P += g->e_shared[k] ? g->e_ncfg[k] : (int64_t)g->e_ncfg[k] * g->e_nfac[k];
    double *hist = (double *)calloc((size_t)(n_iters + 1) * (size_t)(ES > 0 ? ES : 1), sizeof(double));
    double *v2f = (double *)malloc(sizeof(double) * (size_t)(ES > 0 ? ES : 1));
    double *mt = (double *)malloc(sizeof(double) * (size_t)(ES > 0 ? ES : 1));
    double *dm = (double *)calloc((size_t)(ES > 0 ? ES : 1), sizeof(double));
    double *dm_prev = (double *)calloc((size_t)(ES > 0 ? ES : 1), sizeof(double));
    double *dv = (double *)calloc((size_t)(ES > 0 ? ES : 1), sizeof(double));
    double *vals = (double *)malloc(sizeof(double) * (size_t)max_ncfg(g));
    uint32_t fl = 0;
    /* forward, keeping every message state */
    for (int t = 1; t <= n_iters; ++t) {
        const double *mo = hist + (size_t)(t - 1) * ES;
        double *mn = hist + (size_t)t * ES;
        var_to_factor(g, &L, evidence, mo, v2f);
        for (int k = 0; k < g->n_enum; ++k)
            for (int64_t f = 0; f < g->e_nfac[k]; ++f) enum_factor(g, &L, k, f, log_pot, T, v2f, mt, vals);
        for (int k = 0; k < g->n_logic; ++k)
            for (int64_t f = 0; f < g->l_nfac[k]; ++f) {
                const int32_t *po = g->l_paroff[k];
                int64_t s0 = L.es_off[L.logic_edge0[k] + po[f] + f];
                logic_closed(g->l_kind[k], po[f + 1] - po[f], v2f + s0, T, mt + s0);
            }
        for (int64_t e = 0; e < L.E; ++e) {
            int K = (int)(L.es_off[e + 1] - L.es_off[e]);
            damp_normalise(mt + L.es_off[e], mo + L.es_off[e], K, damping, &fl);
        }
        memcpy(mn, mt, sizeof(double) * (size_t)ES);
    }
    for (int64_t i = 0; i < P; ++i) d_log_pot[i] = 0.0;
    for (int64_t i = 0; i < VS; ++i) d_evidence[i] = 0.0;
    /* beliefs: db = g - softmax(b) sum(g); de += db; dm_e = db_{v(e)} */
    {
        const double *mfin = hist + (size_t)n_iters * ES;
        for (int64_t v = 0; v < L.V; ++v) {
            int K = g->num_states[v];
            double b[PGM_ORACLE_KMAX], sg = 0.0;
            for (int x = 0; x < K; ++x) {
                double s = evidence[L.vs_off[v] + x];
                for (int64_t q = L.vin_off[v]; q < L.vin_off[v + 1]; ++q) s += mfin[L.es_off[L.vin_edge[q]] + x];
                b[x] = s;
                sg += g_nb[L.vs_off[v] + x];
            }
            double z = lse_T(b, K, 1.0);
            for (int x = 0; x < K; ++x) {
                double db = g_nb[L.vs_off[v] + x] - exp(b[x] - z) * sg;
                d_evidence[L.vs_off[v] + x] += db;
                for (int64_t q = L.vin_off[v]; q < L.vin_off[v + 1]; ++q) dm[L.es_off[L.vin_edge[q]] + x] = db;
            }
        }
    }
    /* iterations, last to first */
    for (int t = n_iters; t >= 1; --t) {
        const double *mo = hist + (size_t)(t - 1) * ES;
        var_to_factor(g, &L, evidence, mo, v2f);
        for (int k = 0; k < g->n_enum; ++k)
            for (int64_t f = 0; f < g->e_nfac[k]; ++f) enum_factor(g, &L, k, f, log_pot, T, v2f, mt, vals);
        for (int k = 0; k < g->n_logic; ++k)
            for (int64_t f = 0; f < g->l_nfac[k]; ++f) {
                const int32_t *po = g->l_paroff[k];
                int64_t s0 = L.es_off[L.logic_edge0[k] + po[f] + f];
                logic_closed(g->l_kind[k], po[f + 1] - po[f], v2f + s0, T, mt + s0);
            }
        for (int64_t i = 0; i < ES; ++i) {
            dm_prev[i] = 0.0;
            dv[i] = 0.0;
        }
        /* normalise, damp, normalise: backward per edge; dm becomes d(mt) */
        for (int64_t e = 0; e < L.E; ++e) {
            int K = (int)(L.es_off[e + 1] - L.es_off[e]);
            double *me = mt + L.es_off[e];
            const double *mold = mo + L.es_off[e];
            double n[PGM_ORACLE_KMAX], d[PGM_ORACLE_KMAX];
            int a1 = argmax_k(me, K);
            for (int x = 0; x < K; ++x) n[x] = me[x] - me[a1];
            for (int x = 0; x < K; ++x) d[x] = (damping != 0.0) ? damping * mold[x] + (1.0 - damping) * n[x] : n[x];
            int a2 = argmax_k(d, K);
            double *gm = dm + L.es_off[e];
            double sd = 0.0, dd[PGM_ORACLE_KMAX];
            for (int x = 0; x < K; ++x) sd += gm[x];
            for (int x = 0; x < K; ++x) dd[x] = gm[x] - (x == a2 ? sd : 0.0);
            double dn[PGM_ORACLE_KMAX], sn = 0.0;
            for (int x = 0; x < K; ++x) {
                dm_prev[L.es_off[e] + x] += damping * dd[x];
                dn[x] = (damping != 0.0 ? (1.0 - damping) : 1.0) * dd[x];
                sn += dn[x];
            }
            for (int x = 0; x < K; ++x) gm[x] = dn[x] - (x == a1 ? sn : 0.0);
        }
        /* factor backward */
        for (int k = 0; k < g->n_enum; ++k) {
            int a = g->e_arity[k], nc = g->e_ncfg[k];
            const int32_t *cfg = g->e_cfg[k];
            for (int64_t f = 0; f < g->e_nfac[k]; ++f) {
                int64_t e0 = L.enum_edge0[k] + f * a;
                int64_t poff = L.enum_pot0[k] + (g->e_shared[k] ? 0 : f * nc);
                for (int c = 0; c < nc; ++c) {
                    for (int i = 0; i < a; ++i) {
                        double s = log_pot[poff + c];
                        for (int j = 0; j < a; ++j)
                            if (j != i) s += v2f[L.es_off[e0 + j] + cfg[c * a + j]];
                        int64_t ii = L.es_off[e0 + i] + cfg[c * a + i];
                        if (s == -INFINITY) continue;
                        double p = exp((s - mt[ii]) / T);
                        double w = dm[ii] * p;
                        d_log_pot[poff + c] += w;
                        for (int j = 0; j < a; ++j)
                            if (j != i) dv[L.es_off[e0 + j] + cfg[c * a + j]] += w;
                    }
                }
            }
        }
        /* logical factors backward: softmax over the valid configurations */
        for (int k = 0; k < g->n_logic; ++k) {
            const int32_t *po = g->l_paroff[k];
            for (int64_t f = 0; f < g->l_nfac[k]; ++f) {
                int n = po[f + 1] - po[f];
                int64_t s0 = L.es_off[L.logic_edge0[k] + po[f] + f];
                double *raw = (double *)malloc(sizeof(double) * (size_t)(2 * (n + 1)));
                logic_brute(g->l_kind[k], n, v2f + s0, T, raw);
                for (int64_t p = 0; p < ((int64_t)1 << n); ++p) {
                    int any = 0, all = 1;
                    for (int j = 0; j < n; ++j) {
                        any |= (int)((p >> j) & 1);
                        all &= (int)((p >> j) & 1);
                    }
                    int c = logic_child(g->l_kind[k], any, all, p, n);
                    for (int i = 0; i <= n; ++i) {
                        int xi = (i < n) ? (int)((p >> i) & 1) : c;
                        double sv = 0.0;
                        for (int j = 0; j <= n; ++j)
                            if (j != i) sv += v2f[s0 + 2 * j + ((j < n) ? (int)((p >> j) & 1) : c)];
                        if (sv == -INFINITY || raw[2 * i + xi] == -INFINITY) continue;
                        double w = dm[s0 + 2 * i + xi] * exp((sv - raw[2 * i + xi]) / T);
                        for (int j = 0; j <= n; ++j)
                            if (j != i) dv[s0 + 2 * j + ((j < n) ? (int)((p >> j) & 1) : c)] += w;
                    }
                }
                free(raw);
            }
        }
        /* leave-one-out backward: v_{f->v} = e_v + sum_{g != f} m_{g->v} */
        for (int64_t v = 0; v < L.V; ++v) {
            int K = g->num_states[v];
            for (int x = 0; x < K; ++x) {
                double tot = 0.0;
                for (int64_t q = L.vin_off[v]; q < L.vin_off[v + 1]; ++q) tot += dv[L.es_off[L.vin_edge[q]] + x];
                d_evidence[L.vs_off[v] + x] += tot;
                for (int64_t q = L.vin_off[v]; q < L.vin_off[v + 1]; ++q) {
                    int64_t i = L.es_off[L.vin_edge[q]] + x;
                    dm_prev[i] += tot - dv[i];
                }
            }
        }
        memcpy(dm, dm_prev, sizeof(double) * (size_t)ES);
    }
    free(hist);
    free(v2f);
    free(mt);
    free(dm);
    free(dm_prev);
    free(dv);
    free(vals);
    layout_free(&L);
    return 0;
}
