/*
 * grt_oracle.c -- plain, slow, FP64 CPU oracle of the generalized-random-tree
 * point solve of Acebron & Rodriguez-Rozas, "A new parallel solver suited for
 * arbitrary semilinear parabolic partial differential equations based on
 * generalized random trees" (arXiv 2402.06491).
 *
 * TEST INFRASTRUCTURE.  This file is the reference the CUDA path is
 * compared against.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline / reference arm load it.  The product library never links,
 * includes or calls it, and it shares no code, header, table or constant
 * generator with the CUDA path: it has its own Philox, its own threshold
 * tables, its own recursive tree walker and its own Pade solver.
 *
 * What it computes (paper sections / equations):
 *   Problem   u_t = D*Lap(u) + f(u),  u(x,0) = g(x),  f(u) = sum_k b_k u^k
 *             (Sec. 1, Eq. nonlinear_new; Duhamel form Eq. integraleq).
 *   Strategy B  (Sec. 2.2, Eqs. totalduhamel_B, probexpB1, probexpBclosed):
 *             a node is a leaf with probability q and then contributes
 *             g(x + sqrt(2 D tau) n)/q; otherwise it splits at time tau*S,
 *             S ~ U(0,1), with weight eta = tau times b_k/((1-q) p_k), and its
 *             k children start at the split position with remaining time
 *             tau*(1-S).
 *   Strategy A  (Sec. 2.1, Eqs. totalduhamel, probexp1, probexp2, recursion)
 *             generalised to an exponential clock of rate lambda and a
 *             potential c pulled out of f (F(u) = f(u) + c u); lambda = 1,
 *             c = 0 is the paper's u = v e^t change of variables and
 *             c = lambda is McKean's representation (Eq. prod-McK).
 *             Lifetime S = -ln(U)/lambda; S >= tau: leaf with weight
 *             e^{(lambda-c) tau} g(x + sqrt(2 D tau) n); otherwise split at S
 *             with weight e^{(lambda-c) S} b_k/(lambda p_k) and k children at
 *             remaining time tau - S.
 *   Tree walk  The algorithm of Sec. 2.1 (text after Eq. recursion, Fig. 1):
 *             depth-first, children in order, weights multiplied together
 *             (Eq. rep_strategyB / probexpBclosed).
 *   Series    The tree order is its number of splitting events Ne; the
 *             per-order means a_n are the coefficients of the series that is
 *             Pade-summed (Sec. 2.1 end, Sec. 2.4).  Trees with Ne > K are
 *             pruned: they add 0 to every kept order but count in N
 *             (Sec. 2.4, "pruning the trees to kmax").
 *   Pade      [L/M] approximant of sum_n a_n eps^n evaluated at eps = 1
 *             (Sec. 2.1 end, Sec. 2.4), after an eps-rescaling that leaves
 *             the approximant unchanged.
 *   Errors    per-order standard errors (Sec. 2.4, Eq. simplecase_discrete).
 *   General drift and diffusion  L = sum_i (s_i + r_i x_i)^2 / 2 d_ii + (beta_i -
 *             kappa_i x_i) d_i: the segments follow the SDE by Euler-Maruyama
 *             with a fixed number of equal steps per segment (Eqs. SDE, green;
 *             Sec. 2.4 uses the Euler scheme).
 *   Variable coefficients  c_k(x, t) = b_k gamma(x, t) for the terms of a
 *             mask (Sec. 1, Eq. nonlinear_new; Example 5): the split weight
 *             is multiplied by gamma at the split position and at the PDE
 *             time left to the children (Sec. 2.1, Eq. probexp1).
 *
 * Brownian increments.  For L = D*Lap the Green's function (Eqs. green,
 * SDE) is the Gaussian kernel of variance 2 D tau per coordinate, so each
 * path segment is sampled exactly (no time stepping).
 *
 * Random numbers.  Philox4x32-10 of Salmon, Moraes, Dror and Shaw
 * ("Parallel random numbers: as easy as 1, 2, 3", SC'11), written here from
 * that definition.  Every node of every tree draws from its own counter:
 *   key = (seed mod 2^32, seed >> 32)
 *   ctr = (lo32(id), hi32(id), tree | (sub << 31), point)
 * where id is a path label of the node (root 0; child j of node id has label
 * 16*id + j + 1), an analogue of the paper's ancestry labels (Sec. 2.2,
 * Fig. 2), so that the draws do not depend on the traversal order.
 *
 * Word use per node: w0 = node decision (B: joint leaf/term categorical;
 * A: lifetime), w1 = (B: split fraction S; A: term categorical),
 * (w2, w3) = one Box-Muller pair giving normals n0, n1; for d = 3 a second
 * call (sub = 1) gives (w4, w5), a second pair of which n2 is used.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAX_DEG 15
#define OR_MAX_K 16
#define OR_MAX_DIM 3
#define OR_MAX_TERMS 16

/* Mirror of the problem description used by the Python side.  It is a
 * separate struct from the product library's: the two sides share no header. */
typedef struct {
    int32_t dim;
    double D;
    int32_t f_deg;
    double f_coef[OR_MAX_DEG + 1];
    int32_t u0_kind;
    double u0_param[8];
    int32_t strategy; /* 0 = A, 1 = B */
    double lambda;
    double c_pot;
    double q;
    int32_t arity_law; /* 0 = uniform over the terms, 1 = p_k ~ |b_k| */
    int32_t precision; /* unused by the oracle (always FP64); keeps the field order */
    int32_t coef_kind; /* variable coefficients: 0 none, 1 gauss / (t + t0), 2 gauss */
    double coef_param[8];
    uint32_t coef_mask; /* bit k: c_k(x, t) = b_k gamma(x, t) */
    int32_t sde_kind;   /* 0: L = D Lap, exact Gaussian segments; 1: Euler-Maruyama (below) */
    int32_t sde_steps;  /* Euler steps per segment (sde_kind 1) */
    double sde_param[12]; /* beta[3], kappa[3], s[3], r[3] */
} or_problem;

enum { OR_U0_CONST = 0, OR_U0_GAUSS = 1, OR_U0_COS_PROD = 2, OR_U0_TANH_PROD = 3, OR_U0_LOGISTIC = 4,
       OR_U0_GAUSS_AXES = 5, OR_U0_QUADRATIC = 6 };
enum { OR_STRAT_A = 0, OR_STRAT_B = 1 };
enum { OR_COEF_CONST = 0, OR_COEF_GAUSS_OVER_T = 1, OR_COEF_GAUSS = 2 };

enum {
    OR_STATUS_PADE_SINGULAR = 1,
    OR_STATUS_PADE_POLE_NEAR = 2,
    OR_STATUS_SERIES_PARTIAL = 4,
    OR_STATUS_HIGH_PRUNE = 8
};

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32->64 bit      */
/* multiplies with the round constants, the key bumped by the Weyl constants */
/* after every round.                                                        */
/* ------------------------------------------------------------------------ */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform on (0,1) from a 32-bit word: the top 23 bits plus one half,
 * times 2^-23.  Exact in binary32 and binary64, never 0 or 1. */
double oracle_uniform(uint32_t w)
{
    return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* ------------------------------------------------------------------------ */
/* Problem set-up: the terms of the branching law and their thresholds.     */
/* ------------------------------------------------------------------------ */
typedef struct {
    or_problem pb;
    int nterms;
    int arity[OR_MAX_TERMS];       /* power k of each term (ascending k)     */
    double coef[OR_MAX_TERMS];     /* b_k of F (A) or f (B)                  */
    uint64_t thr[OR_MAX_TERMS + 1];/* cumulative u32 thresholds, last = 2^32 */
    int ncat;                      /* number of categories of the draw       */
    double leaf_factor;            /* B: 1 / P(leaf)                         */
    double term_factor[OR_MAX_TERMS]; /* B: b_k/P(k);  A: b_k/(lambda P(k))  */
} or_setup;

static uint64_t or_round_threshold(double cum)
{
    double v = cum * 4294967296.0;
    if (v <= 0.0) return 0;
    if (v >= 4294967296.0) return 4294967296ull;
    return (uint64_t)llround(v);
}

/* Returns 0 on success, -1 on an invalid problem. */
static int or_build_setup(const or_problem *pb, or_setup *s)
{
    memset(s, 0, sizeof(*s));
    s->pb = *pb;
    if (pb->dim < 1 || pb->dim > OR_MAX_DIM) return -1;
    if (pb->f_deg < 0 || pb->f_deg > OR_MAX_DEG) return -1;
    if (!(pb->D >= 0.0)) return -1;
    if (pb->coef_kind < OR_COEF_CONST || pb->coef_kind > OR_COEF_GAUSS) return -1;
    if (pb->sde_kind < 0 || pb->sde_kind > 1) return -1;
    if (pb->sde_kind == 1 && (pb->sde_steps < 1 || pb->sde_steps > 4096)) return -1;
    if (pb->coef_kind == OR_COEF_GAUSS_OVER_T && !(pb->coef_param[6] > 0.0)) return -1;
    /* A variable linear coefficient cannot be combined with a pulled-out
     * constant potential: F's linear coefficient b_1 gamma + c is not b gamma. */
    if (pb->coef_kind != OR_COEF_CONST && pb->strategy == OR_STRAT_A && pb->c_pot != 0.0 &&
        ((pb->coef_mask >> 1) & 1u))
        return -1;
    /* Terms: nonzero coefficients of F = f + c u (A) or f (B), ascending k. */
    for (int k = 0; k <= pb->f_deg; ++k) {
        double b = pb->f_coef[k];
        if (pb->strategy == OR_STRAT_A && k == 1) b += pb->c_pot;
        if (b != 0.0) {
            s->arity[s->nterms] = k;
            s->coef[s->nterms] = b;
            s->nterms++;
        }
    }
    if (pb->strategy == OR_STRAT_A && pb->f_deg < 1 && pb->c_pot != 0.0) {
        s->arity[s->nterms] = 1;
        s->coef[s->nterms] = pb->c_pot;
        s->nterms++;
    }
    /* Branching law p_k over the terms: uniform (the paper's choice, Sec. 2.1
     * after Eq. probexp2) or proportional to |b_k|. */
    double p[OR_MAX_TERMS];
    double sabs = 0.0;
    for (int i = 0; i < s->nterms; ++i) sabs += fabs(s->coef[i]);
    for (int i = 0; i < s->nterms; ++i)
        p[i] = (pb->arity_law == 1) ? fabs(s->coef[i]) / sabs : 1.0 / (double)s->nterms;

    if (pb->strategy == OR_STRAT_B) {
        if (!(pb->q > 0.0 && pb->q < 1.0)) return -1;
        if (s->nterms == 0) {
            /* f = 0: every node is a leaf. */
            s->ncat = 1;
            s->thr[0] = 4294967296ull;
            s->leaf_factor = 1.0;
            return 0;
        }
        /* Joint categorical over {leaf, term 1, ..., term n}:
         * P(leaf) = q, P(term i) = (1-q) p_i.  Thresholds
         * T_0 = round(2^32 q), T_j = round(2^32 (q + (1-q) sum_{i<=j} p_i)). */
        s->ncat = s->nterms + 1;
        s->thr[0] = or_round_threshold(pb->q);
        double cp = 0.0;
        for (int i = 0; i < s->nterms; ++i) {
            cp += p[i];
            s->thr[i + 1] = or_round_threshold(pb->q + (1.0 - pb->q) * cp);
        }
        s->thr[s->nterms] = 4294967296ull;
        /* Weights use the probabilities the thresholds realise exactly. */
        s->leaf_factor = 4294967296.0 / (double)s->thr[0];
        for (int i = 0; i < s->nterms; ++i) {
            double P = (double)(s->thr[i + 1] - s->thr[i]) / 4294967296.0;
            s->term_factor[i] = (P > 0.0) ? s->coef[i] / P : 0.0;
        }
    } else {
        if (!(pb->lambda > 0.0)) return -1;
        if (s->nterms == 0) {
            s->ncat = 0;
            return 0;
        }
        s->ncat = s->nterms;
        double cp = 0.0;
        for (int i = 0; i < s->nterms; ++i) {
            cp += p[i];
            s->thr[i] = or_round_threshold(cp);
        }
        s->thr[s->nterms - 1] = 4294967296ull;
        for (int i = 0; i < s->nterms; ++i) {
            uint64_t lo = (i == 0) ? 0 : s->thr[i - 1];
            double P = (double)(s->thr[i] - lo) / 4294967296.0;
            s->term_factor[i] = (P > 0.0) ? s->coef[i] / (pb->lambda * P) : 0.0;
        }
    }
    return 0;
}

/* Smallest category j with w < thr[j]. */
static int or_draw_category(const or_setup *s, uint32_t w)
{
    for (int j = 0; j < s->ncat; ++j)
        if ((uint64_t)w < s->thr[j]) return j;
    return s->ncat - 1;
}

/* Initial data g(x). */
static double or_u0(const or_problem *pb, const double *x)
{
    const double *a = pb->u0_param;
    int d = pb->dim;
    switch (pb->u0_kind) {
    case OR_U0_CONST:
        return a[0];
    case OR_U0_GAUSS: { /* a0 + a1 exp(-|x - x0|^2 / (2 a2^2)), x0 = (a3, a4, a5) */
        double r2 = 0.0;
        for (int i = 0; i < d; ++i) {
            double e = x[i] - a[3 + i];
            r2 += e * e;
        }
        return a[0] + a[1] * exp(-r2 / (2.0 * a[2] * a[2]));
    }
    case OR_U0_COS_PROD: { /* a0 + a1 prod_i cos(a[2+i] x_i) */
        double pr = 1.0;
        for (int i = 0; i < d; ++i) pr *= cos(a[2 + i] * x[i]);
        return a[0] + a[1] * pr;
    }
    case OR_U0_TANH_PROD: { /* a0 + a1 prod_i tanh(x_i - a[2+i]) */
        double pr = 1.0;
        for (int i = 0; i < d; ++i) pr *= tanh(x[i] - a[2 + i]);
        return a[0] + a[1] * pr;
    }
    case OR_U0_LOGISTIC: /* a0 + a1 / (1 + exp(-(x_0 - a2) / a3)) */
        return a[0] + a[1] / (1.0 + exp(-(x[0] - a[2]) / a[3]));
    case OR_U0_QUADRATIC: { /* a0 + sum_i (a[1+i] x_i + a[4+i] x_i^2) */
        double v = a[0];
        for (int i = 0; i < d; ++i) v += a[1 + i] * x[i] + a[4 + i] * x[i] * x[i];
        return v;
    }
    case OR_U0_GAUSS_AXES: { /* a0 + a1 exp(-sum_i a[2+i] (x_i - a[5+i])^2) */
        double r = 0.0;
        for (int i = 0; i < d; ++i) {
            double e = x[i] - a[5 + i];
            r += a[2 + i] * e * e;
        }
        return a[0] + a[1] * exp(-r);
    }
    default:
        return NAN;
    }
}

/* Variable-coefficient profile gamma(x, t) of the terms selected by the mask,
 * c_k(x, t) = b_k gamma(x, t) (Sec. 1, Eq. nonlinear_new: f = sum_j c_j(x,t) u^j):
 *   GAUSS_OVER_T  exp(-sum_i a_i (x_i - a_{3+i})^2) / (t + a6)   (Example 5 shape)
 *   GAUSS         exp(-sum_i a_i (x_i - a_{3+i})^2)
 * t is the PDE time at which the term acts. */
static double or_gamma(const or_problem *pb, const double *x, double t)
{
    const double *a = pb->coef_param;
    double r = 0.0;
    for (int i = 0; i < pb->dim; ++i) {
        double e = x[i] - a[3 + i];
        r += a[i] * e * e;
    }
    double g = exp(-r);
    if (pb->coef_kind == OR_COEF_GAUSS_OVER_T) g /= (t + a[6]);
    return g;
}

/* ------------------------------------------------------------------------ */
/* One tree, walked recursively.                                            */
/* ------------------------------------------------------------------------ */
typedef struct {
    const or_setup *s;
    uint32_t key[2];
    uint32_t tree, point;
    int K;
    int Ne;          /* splitting events so far */
    int pruned;      /* Ne exceeded K           */
    uint32_t nodes;  /* nodes visited           */
    double W;        /* running product         */
    uint64_t hash;   /* FNV-1a over node codes in preorder */
} or_tree;

static void or_hash_code(or_tree *T, uint64_t code)
{
    T->hash ^= code;
    T->hash *= 0x100000001B3ull;
}

/* Euler-Maruyama for dX_i = (beta_i - kappa_i X_i) dt + (s_i + r_i X_i) dW_i over a
 * segment of length s_seg (Eqs. SDE, green: the paths of a general operator L
 * = a_ij d_i d_j + b_i d_i with sigma^2 = a, simulated by the Euler scheme as
 * in Sec. 2.4).  A fixed number m = sde_steps of equal steps h = s_seg / m.
 * Normals come from Philox blocks at the node's counter with the sub bit set,
 * block b under the key (k0 ^ (b+1) 0x2545F491, k1 ^ (b+1) 0x6C8E9CF5), each
 * Box-Muller pair (u, v) giving r cos(2 pi v), r sin(2 pi v), r = sqrt(-2 ln u):
 *   d <= 2: block b serves steps 2b (pair (w0, w1)) and 2b + 1 (pair (w2, w3));
 *   d = 3:  block b serves step b: (w0, w1) -> n0, n1 and (w2, w3) -> n2 (cos). */
static void or_bm_pair(uint32_t wu, uint32_t wv, double *z0, double *z1)
{
    double r = sqrt(-2.0 * log(oracle_uniform(wu)));
    double a = 2.0 * M_PI * oracle_uniform(wv);
    *z0 = r * cos(a);
    *z1 = r * sin(a);
}

static void or_euler_segment(const or_tree *T, const or_problem *pb, const double *x, double s_seg, uint64_t id,
                             double *y)
{
    const double *beta = pb->sde_param, *kappa = pb->sde_param + 3, *sd = pb->sde_param + 6,
                 *rr = pb->sde_param + 9;
    int d = pb->dim;
    int m = pb->sde_steps;
    double h = s_seg / (double)m, sh = sqrt(h);
    for (int i = 0; i < d; ++i) y[i] = x[i];
    uint32_t w[4] = { 0, 0, 0, 0 };
    for (int j = 0; j < m; ++j) {
        int b = (d <= 2) ? j / 2 : j;
        int first = (d <= 2) ? (j % 2 == 0) : 1;
        if (first) {
            uint32_t bb = (uint32_t)(b + 1);
            uint32_t key[2] = { T->key[0] ^ (bb * 0x2545F491u), T->key[1] ^ (bb * 0x6C8E9CF5u) };
            uint32_t ctr[4] = { (uint32_t)id, (uint32_t)(id >> 32), T->tree | 0x80000000u, T->point };
            oracle_philox4x32_10(ctr, key, w);
        }
        double z[3], dummy;
        if (d <= 2) {
            if (j % 2 == 0) or_bm_pair(w[0], w[1], &z[0], &z[1]);
            else or_bm_pair(w[2], w[3], &z[0], &z[1]);
            z[2] = 0.0;
        } else {
            or_bm_pair(w[0], w[1], &z[0], &z[1]);
            or_bm_pair(w[2], w[3], &z[2], &dummy);
        }
        for (int i = 0; i < d; ++i) {
            double X = y[i];
            y[i] = X + (beta[i] - kappa[i] * X) * h + (sd[i] + rr[i] * X) * sh * z[i];
        }
    }
}

static void or_visit(or_tree *T, const double *x, double tau, uint64_t id)
{
    const or_setup *s = T->s;
    const or_problem *pb = &s->pb;
    int d = pb->dim;
    T->nodes++;

    uint32_t ctr[4] = { (uint32_t)id, (uint32_t)(id >> 32), T->tree, T->point };
    uint32_t w[8];
    oracle_philox4x32_10(ctr, T->key, w);
    if (d == 3) {
        uint32_t ctr1[4] = { ctr[0], ctr[1], T->tree | 0x80000000u, T->point };
        oracle_philox4x32_10(ctr1, T->key, w + 4);
    }
    /* Box-Muller normals. */
    double n[3];
    {
        double r = sqrt(-2.0 * log(oracle_uniform(w[2])));
        double ang = 2.0 * M_PI * oracle_uniform(w[3]);
        n[0] = r * cos(ang);
        n[1] = r * sin(ang);
        if (d == 3) {
            double r2 = sqrt(-2.0 * log(oracle_uniform(w[4])));
            n[2] = r2 * cos(2.0 * M_PI * oracle_uniform(w[5]));
        }
    }

    int leaf;
    int cat = -1;       /* index of the chosen term */
    double s_seg;       /* duration of this node's Brownian segment */
    double tau_child = 0.0;
    double factor;
    if (pb->strategy == OR_STRAT_B) {
        int c = or_draw_category(s, w[0]);
        leaf = (c == 0);
        if (leaf) {
            s_seg = tau;
            factor = s->leaf_factor;
        } else {
            cat = c - 1;
            double S = oracle_uniform(w[1]);
            s_seg = tau * S;
            tau_child = tau * (1.0 - S);
            factor = tau * s->term_factor[cat];
        }
    } else {
        double S = -log(oracle_uniform(w[0])) / pb->lambda;
        leaf = (S >= tau) || (s->ncat == 0);
        if (leaf) {
            s_seg = tau;
            /* With no term (f = 0, hence c = 0) there is no clock: u = E[g], weight g. */
            factor = (s->ncat == 0) ? 1.0 : exp((pb->lambda - pb->c_pot) * tau);
        } else {
            cat = or_draw_category(s, w[1]);
            s_seg = S;
            tau_child = tau - S;
            factor = exp((pb->lambda - pb->c_pot) * S) * s->term_factor[cat];
        }
    }

    double y[OR_MAX_DIM];
    if (pb->sde_kind == 1) {
        or_euler_segment(T, pb, x, s_seg, id, y);
    } else {
        double sc = sqrt(2.0 * pb->D * s_seg);
        for (int i = 0; i < d; ++i) y[i] = x[i] + sc * n[i];
    }

    if (leaf) {
        or_hash_code(T, 0);
        T->W *= factor * or_u0(pb, y);
        return;
    }
    or_hash_code(T, (uint64_t)(cat + 1));
    T->Ne++;
    if (T->Ne > T->K) {
        T->pruned = 1;
        return;
    }
    int k = s->arity[cat];
    /* A variable coefficient acts where and when the particle splits: at the
     * end y of this segment and at PDE time tau_child, the time left to its
     * children (Sec. 2.1, Eq. probexp1: c_j(beta(S), t - S)). */
    if (pb->coef_kind != OR_COEF_CONST && ((pb->coef_mask >> k) & 1u)) factor *= or_gamma(pb, y, tau_child);
    T->W *= factor;
    for (int j = 0; j < k; ++j) {
        or_visit(T, y, tau_child, 16ull * id + (uint64_t)j + 1ull);
        if (T->pruned) return;
    }
}

static void or_walk_tree(const or_setup *s, uint64_t seed, uint32_t point, uint32_t tree,
                         const double *x, double t, int K, or_tree *T)
{
    T->s = s;
    T->key[0] = (uint32_t)seed;
    T->key[1] = (uint32_t)(seed >> 32);
    T->tree = tree;
    T->point = point;
    T->K = K;
    T->Ne = 0;
    T->pruned = 0;
    T->nodes = 0;
    T->W = 1.0;
    T->hash = 0xCBF29CE484222325ull;
    or_visit(T, x, t, 0ull);
}

/* Per-tree records for a tree range of one point: order (Ne, or K+1 when
 * pruned), weight (0 when pruned), nodes visited, topology hash. */
int oracle_trees(const or_problem *pb, const double *x, double t, uint64_t point_index,
                 uint64_t first_tree, uint64_t ntrees, int K, uint64_t seed,
                 int32_t *order, double *w, uint32_t *nodes, uint64_t *hash)
{
    or_setup s;
    if (or_build_setup(pb, &s) != 0) return -1;
    if (K < 0 || K > OR_MAX_K) return -1;
    if (first_tree + ntrees > 0x80000000ull || point_index > 0xFFFFFFFFull) return -1;
    for (uint64_t i = 0; i < ntrees; ++i) {
        or_tree T;
        or_walk_tree(&s, seed, (uint32_t)point_index, (uint32_t)(first_tree + i), x, t, K, &T);
        if (order) order[i] = T.pruned ? K + 1 : T.Ne;
        if (w) w[i] = T.pruned ? 0.0 : T.W;
        if (nodes) nodes[i] = T.nodes;
        if (hash) hash[i] = T.hash;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* [L/M] Pade approximant at eps = 1 (Sec. 2.1 end, Sec. 2.4).              */
/*   Denominator: beta_0 = 1, sum_{j=1..M} c_{L+i-j} beta_j = -c_{L+i},     */
/*   i = 1..M (c_{<0} = 0); numerator alpha_i = sum_{j<=min(i,M)} beta_j    */
/*   c_{i-j}.  Solved on c_n = a_n / rho^n and evaluated at w = rho, which  */
/*   equals the unscaled approximant at eps = 1 (a Pade approximant is      */
/*   invariant under eps -> s eps; the paper fixes no scaling; rho is a     */
/*   power of two, so the rescaling itself is exact).  A pivot below 1e-14  */
/*   times the largest matrix entry lowers the type to [L-1/M-1] (L stays   */
/*   >= 0).                                                                 */
/* ------------------------------------------------------------------------ */
int oracle_pade(int L, int M, const double *a, double *u_out, int32_t *status_out, int32_t *lm_used)
{
    int32_t status = 0;
    if (L < 0 || M < 0 || L + M > OR_MAX_K) return -1;
    int n = L + M;
    /* Scale: rho = 2^k with k the integer growth rate of the binary exponents,
     * k = max_{j > m} ceil((e_j - e_m) / (j - m)), e_j = ilogb(a_j), m the first
     * nonzero coefficient: a root-test estimate rounded to a power of two, so
     * that c_j = a_j 2^{-k j} is exact and |c_j| < 2^{e_m - k m + 1}.  k = 0 when
     * no two coefficients are nonzero. */
    int m = 0;
    while (m <= n && a[m] == 0.0) ++m;
    int k = 0, have = 0;
    for (int j = m + 1; j <= n; ++j)
        if (a[j] != 0.0) {
            int num = ilogb(a[j]) - ilogb(a[m]), den = j - m;
            int q = num / den;
            if (num % den != 0 && num > 0) q += 1; /* ceiling for positive, C truncation is the ceiling for negative */
            if (!have || q > k) k = q;
            have = 1;
        }
    double rho = ldexp(1.0, k);
    double c[OR_MAX_K + 1];
    for (int i = 0; i <= n; ++i) c[i] = ldexp(a[i], -k * i);
    int Lc = L, Mc = M;
    double beta[OR_MAX_K + 1];
    for (;;) {
        beta[0] = 1.0;
        if (Mc == 0) break;
        /* Build the Mc x Mc Toeplitz system A beta = rhs. */
        double A[OR_MAX_K][OR_MAX_K + 1];
        double amax = 0.0;
        for (int i = 1; i <= Mc; ++i) {
            for (int j = 1; j <= Mc; ++j) {
                int idx = Lc + i - j;
                A[i - 1][j - 1] = (idx >= 0) ? c[idx] : 0.0;
                if (fabs(A[i - 1][j - 1]) > amax) amax = fabs(A[i - 1][j - 1]);
            }
            A[i - 1][Mc] = -c[Lc + i];
        }
        /* Gaussian elimination with partial pivoting. */
        int singular = (amax == 0.0);
        for (int col = 0; col < Mc && !singular; ++col) {
            int piv = col;
            for (int r = col + 1; r < Mc; ++r)
                if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
            if (fabs(A[piv][col]) <= 1e-14 * amax) {
                singular = 1;
                break;
            }
            if (piv != col)
                for (int j = 0; j <= Mc; ++j) {
                    double tmp = A[col][j];
                    A[col][j] = A[piv][j];
                    A[piv][j] = tmp;
                }
            for (int r = col + 1; r < Mc; ++r) {
                double m = A[r][col] / A[col][col];
                for (int j = col; j <= Mc; ++j) A[r][j] -= m * A[col][j];
            }
        }
        if (!singular) {
            for (int i = Mc - 1; i >= 0; --i) {
                double acc = A[i][Mc];
                for (int j = i + 1; j < Mc; ++j) acc -= A[i][j] * beta[j + 1];
                beta[i + 1] = acc / A[i][i];
            }
            break;
        }
        status |= OR_STATUS_PADE_SINGULAR;
        Mc -= 1;
        if (Lc > 0) Lc -= 1;
    }
    /* Evaluate P(rho) and Q(rho) by Horner. */
    double Q = 0.0;
    for (int j = Mc; j >= 0; --j) Q = Q * rho + beta[j];
    double P = 0.0;
    for (int i = Lc; i >= 0; --i) {
        double al = 0.0;
        for (int j = 0; j <= (i < Mc ? i : Mc); ++j) al += beta[j] * c[i - j];
        P = P * rho + al;
    }
    if (fabs(Q) < 1e-8) status |= OR_STATUS_PADE_POLE_NEAR;
    *u_out = P / Q;
    if (status_out) *status_out = status;
    if (lm_used) {
        lm_used[0] = Lc;
        lm_used[1] = Mc;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Point solve: N_p trees per point, per-order sums, coefficients, Pade.    */
/* ------------------------------------------------------------------------ */
typedef struct {
    const or_setup *s;
    int64_t n;
    const double *x, *t;
    const uint64_t *ntrees;
    int K, L, M;
    uint64_t seed, point_base;
    int nthreads, tid;
    double *u, *coef, *se;
    int32_t *status;
    double *s1, *s2, *sa;  /* optional raw sums [n][K+1] */
    uint64_t *cnt;         /* optional counts [n][K+2] (K+1 = pruned) */
    uint64_t *nodes;       /* optional [n] */
} or_job;

static void or_solve_point(const or_job *J, int64_t p)
{
    const or_setup *s = J->s;
    int K = J->K, d = s->pb.dim;
    double S1[OR_MAX_K + 1], S2[OR_MAX_K + 1], SA[OR_MAX_K + 1];
    uint64_t C[OR_MAX_K + 2];
    uint64_t nodes = 0;
    for (int i = 0; i <= K; ++i) S1[i] = S2[i] = SA[i] = 0.0;
    for (int i = 0; i <= K + 1; ++i) C[i] = 0;
    uint64_t N = J->ntrees[p];
    const double *xp = J->x + (size_t)p * (size_t)d;
    uint32_t point = (uint32_t)(J->point_base + (uint64_t)p);
    for (uint64_t i = 0; i < N; ++i) {
        or_tree T;
        or_walk_tree(s, J->seed, point, (uint32_t)i, xp, J->t[p], K, &T);
        nodes += T.nodes;
        if (T.pruned) {
            C[K + 1]++;
            continue;
        }
        S1[T.Ne] += T.W;
        S2[T.Ne] += T.W * T.W;
        SA[T.Ne] += fabs(T.W);
        C[T.Ne]++;
    }
    /* Coefficients a_n = S1/N and standard errors (Sec. 2.4). */
    double a[OR_MAX_K + 1], se[OR_MAX_K + 1];
    for (int i = 0; i <= K; ++i) {
        a[i] = (N > 0) ? S1[i] / (double)N : 0.0;
        double var = (N > 1) ? (S2[i] / (double)N - a[i] * a[i]) / (double)(N - 1) : 0.0;
        se[i] = var > 0.0 ? sqrt(var) : 0.0;
    }
    double u = 0.0;
    int32_t st = 0;
    oracle_pade(J->L, J->M, a, &u, &st, NULL);
    if (N > 0 && (double)C[K + 1] > 0.01 * (double)N) st |= OR_STATUS_HIGH_PRUNE;
    J->u[p] = u;
    if (J->status) J->status[p] = st;
    for (int i = 0; i <= K; ++i) {
        size_t o = (size_t)p * (size_t)(K + 1) + (size_t)i;
        if (J->coef) J->coef[o] = a[i];
        if (J->se) J->se[o] = se[i];
        if (J->s1) J->s1[o] = S1[i];
        if (J->s2) J->s2[o] = S2[i];
        if (J->sa) J->sa[o] = SA[i];
    }
    if (J->cnt)
        for (int i = 0; i <= K + 1; ++i) J->cnt[(size_t)p * (size_t)(K + 2) + (size_t)i] = C[i];
    if (J->nodes) J->nodes[p] = nodes;
}

static void *or_worker(void *arg)
{
    const or_job *J = (const or_job *)arg;
    for (int64_t p = J->tid; p < J->n; p += J->nthreads) or_solve_point(J, p);
    return NULL;
}

/* Solve n points.  Points are spread over nthreads host threads (point p
 * goes to thread p mod nthreads); results do not depend on nthreads. */
int oracle_solve(const or_problem *pb, int64_t n, const double *x, const double *t,
                 const uint64_t *ntrees, int K, int L, int M, uint64_t seed, uint64_t point_base,
                 int nthreads, double *u, double *coef, double *se, int32_t *status, double *s1,
                 double *s2, double *sa, uint64_t *cnt, uint64_t *nodes)
{
    or_setup s;
    if (or_build_setup(pb, &s) != 0) return -1;
    if (K < 0 || K > OR_MAX_K || L < 0 || M < 0 || L + M > K) return -1;
    for (int64_t p = 0; p < n; ++p) {
        if (ntrees[p] > 0x80000000ull) return -1;
        if (point_base + (uint64_t)p > 0xFFFFFFFFull) return -1;
        if (!(t[p] >= 0.0)) return -1;
    }
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 1024) nthreads = 1024;
    if ((int64_t)nthreads > n) nthreads = (int)(n > 0 ? n : 1);
    or_job base = { &s, n, x, t, ntrees, K, L, M, seed, point_base, nthreads, 0,
                    u, coef, se, status, s1, s2, sa, cnt, nodes };
    if (nthreads == 1) {
        or_worker(&base);
        return 0;
    }
    pthread_t th[1024];
    or_job jobs[1024];
    int started = 0;
    for (int i = 0; i < nthreads; ++i) {
        jobs[i] = base;
        jobs[i].tid = i;
        if (pthread_create(&th[i], NULL, or_worker, &jobs[i]) != 0) break;
        started++;
    }
    for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
    /* Any thread that failed to start: run its share here. */
    for (int i = started; i < nthreads; ++i) or_worker(&jobs[i]);
    return 0;
}

/* Expose the branching-law tables (for the tests of the law itself). */
int oracle_setup_tables(const or_problem *pb, int32_t *nterms, int32_t *arity, double *coef,
                        uint64_t *thr, double *leaf_factor, double *term_factor)
{
    or_setup s;
    if (or_build_setup(pb, &s) != 0) return -1;
    *nterms = s.nterms;
    for (int i = 0; i < s.nterms; ++i) {
        arity[i] = s.arity[i];
        coef[i] = s.coef[i];
        term_factor[i] = s.term_factor[i];
    }
    for (int i = 0; i < s.ncat; ++i) thr[i] = s.thr[i];
    *leaf_factor = s.leaf_factor;
    return s.ncat;
}

double oracle_u0(const or_problem *pb, const double *x) { return or_u0(pb, x); }
