/*
 * oracle.c -- plain FP64 CPU value iteration, policy evaluation and rollouts
 * for the perishable inventory MDP (Farrington et al. 2023).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  Nothing here is
 * shared with the CUDA library.
 *
 * Everything is computed the slow, obvious way:
 *   - the transition T(s, a, omega) is the paper's closed-form issuing
 *     equations (Eq. demoor:fifo, Eq. demoor:lifo) evaluated per outcome;
 *   - the reward is Eq. demoor:reward (plus revenue per unit issued, the
 *     Scenario B reward) evaluated per outcome, not from expectation tables;
 *   - Q(s, a) = sum over outcomes of P(omega) [r + gamma V(s')] in the order
 *     d (then d2, then u) ascending (Eq. valueiterationdetupdate);
 *   - V_i(s) = max_a Q(s, a); policy = first argmax (Eq. valueiterationdetpolicy,
 *     Algorithm 1 extraction step);
 *   - stopping: span of V_i - V_{i-1} (Scenario B convergence test) or its
 *     sup-norm (Scenario A convergence test), strictly below tol.
 * Build with -ffp-contract=off so that no multiply-add is fused.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXDIG 48

static int valid(const orc_problem *P);
static int ipos(int x) { return x > 0 ? x : 0; }
static int imin(int a, int b) { return a < b ? a : b; }

static long long ipow(long long b, int e) {
    long long r = 1;
    for (int i = 0; i < e; ++i) r *= b;
    return r;
}

static long long product_states(const orc_problem *P, int k) {
    return ipow(P->Q[k] + 1, (P->m[k] - 1) + (P->L[k] - 1));
}

long long orc_num_states(const orc_problem *P) {
    long long n = product_states(P, 0);
    if (P->n_products == 2) n *= product_states(P, 1);
    return n;
}

int orc_num_actions(const orc_problem *P) {
    int n = P->Q[0] + 1;
    if (P->n_products == 2) n *= P->Q[1] + 1;
    return n;
}

typedef struct {
    long long s_next;   /* next product-state index */
    int total;          /* T: units available for issuing (on hand + arrival) */
    int issued, wasted, carried, shortage, arrived;
} prod_out;

/*
 * One product, one period.  s = product state, a = order placed now,
 * z = demand facing this product.  Y_1..Y_{m-1} = X_1..X_{m-1}, Y_m = arrival.
 */
static void product_step(int m, int L, int Q, int issuing, long long s, int a, int z, prod_out *o) {
    int K = (m - 1) + (L - 1);
    int dig[MAXDIG];
    long long rem = s;
    for (int k = 0; k < K; ++k) {
        dig[k] = (int)(rem % (Q + 1));
        rem /= (Q + 1);
    }
    int Y[MAXDIG + 2];                         /* 1-based */
    for (int j = 1; j <= m - 1; ++j) Y[j] = dig[j - 1];
    int arrival = (L >= 2) ? dig[m - 1] : a;   /* P_1 arrives now; with L = 1 the order itself */
    Y[m] = arrival;
    int T = 0;
    for (int j = 1; j <= m; ++j) T += Y[j];

    int Xn[MAXDIG + 2];
    int W;
    if (issuing == 0) {
        /* FIFO, Eq. demoor:fifo: W = [Y_1 - D]^+, X'_j = [Y_{j+1} - [D - sum_{k<=j} Y_k]^+]^+ */
        W = ipos(Y[1] - z);
        for (int j = 1; j <= m - 1; ++j) {
            int cum = 0;
            for (int k = 1; k <= j; ++k) cum += Y[k];
            Xn[j] = ipos(Y[j + 1] - ipos(z - cum));
        }
    } else {
        /* LIFO, Eq. demoor:lifo: W = [Y_1 - [D - sum_{k=2}^m Y_k]^+]^+,
           X'_j = [Y_{j+1} - [D - sum_{k=j+2}^m Y_k]^+]^+ */
        int tail = 0;
        for (int k = 2; k <= m; ++k) tail += Y[k];
        W = ipos(Y[1] - ipos(z - tail));
        for (int j = 1; j <= m - 1; ++j) {
            int t2 = 0;
            for (int k = j + 2; k <= m; ++k) t2 += Y[k];
            Xn[j] = ipos(Y[j + 1] - ipos(z - t2));
        }
    }
    /* pipeline: P'_k = P_{k+1}, P'_{L-1} = a (the order placed now) */
    long long sn = 0, w = 1;
    for (int j = 1; j <= m - 1; ++j) { sn += (long long)Xn[j] * w; w *= (Q + 1); }
    for (int k = 1; k <= L - 1; ++k) {
        int pk = (k <= L - 2) ? dig[m - 1 + k] : a;
        sn += (long long)pk * w;
        w *= (Q + 1);
    }
    o->s_next = sn;
    o->total = T;
    o->issued = imin(z, T);
    o->wasted = W;
    o->carried = ipos(T - z - W);   /* [X_t - D_t - W_t]^+ of Eq. demoor:reward */
    o->shortage = ipos(z - T);
    o->arrived = arrival;
}

static double binom_pmf_direct(int n, int k, double rho) {
    /* C(n, k) rho^k (1 - rho)^(n - k); n <= 60 so C(n,k) is exact in double */
    double c = 1.0;
    for (int i = 1; i <= k; ++i) c = c * (double)(n - k + i) / (double)i;
    return c * pow(rho, (double)k) * pow(1.0 - rho, (double)(n - k));
}

/* the same values, tabulated once per rho (pow is the slow part of the loop) */
#define BINOM_N 64
static double g_binom[BINOM_N + 1][BINOM_N + 1];
static double g_binom_rho = -1.0;

static void ensure_binom(const orc_problem *P) {
    if (P->n_products != 2 || g_binom_rho == P->rho) return;
    for (int n = 0; n <= BINOM_N; ++n)
        for (int k = 0; k <= n; ++k) g_binom[n][k] = binom_pmf_direct(n, k, P->rho);
    g_binom_rho = P->rho;
}

static double binom_pmf(int n, int k, double rho) {
    if (n <= BINOM_N && rho == g_binom_rho) return g_binom[n][k];
    return binom_pmf_direct(n, k, rho);
}

int orc_transition(const orc_problem *P, long long s, int a, int d1, int d2, int u, orc_step *out) {
    if (P->n_products == 1) {
        prod_out o;
        product_step(P->m[0], P->L[0], P->Q[0], P->issuing, s, a, d1, &o);
        const double *c = P->cost[0];
        double r = 0.0;
        r -= c[0] * (double)a;
        r -= c[1] * (double)o.carried;
        r -= c[2] * (double)o.shortage;
        r -= c[3] * (double)o.wasted;
        r += c[4] * (double)o.issued;
        out->s_next = o.s_next;
        out->reward = r;
        out->demand = d1;
        out->issued = o.issued;
        out->wasted = o.wasted;
        out->carried = o.carried;
        out->arrived = o.arrived;
        out->shortage = o.shortage;
        out->unmet1 = o.shortage;
        out->demand_k[0] = d1;
        out->issued_k[0] = o.issued;
        out->wasted_k[0] = o.wasted;
        out->carried_k[0] = o.carried;
        out->arrived_k[0] = o.arrived;
        out->demand_k[1] = out->issued_k[1] = out->wasted_k[1] = 0.0;
        out->carried_k[1] = out->arrived_k[1] = 0.0;
        out->sub_served = 0;
        return 0;
    }
    long long S1 = product_states(P, 0);
    long long s1 = s % S1, s2 = s / S1;
    int A2 = P->Q[1] + 1;
    int a1 = a / A2, a2 = a % A2;
    prod_out o1, o2;
    product_step(P->m[0], P->L[0], P->Q[0], P->issuing, s1, a1, d1, &o1);
    int unmet1 = o1.shortage;
    if (u > unmet1) return 1;
    /* product 2 serves its own demand, then the u substituting customers */
    product_step(P->m[1], P->L[1], P->Q[1], P->issuing, s2, a2, d2 + u, &o2);
    int own2 = imin(d2, o2.total);
    int sub_served = o2.issued - own2;
    int short1 = unmet1 - sub_served;
    int short2 = ipos(d2 - o2.total);
    const double *c1 = P->cost[0], *c2 = P->cost[1];
    double r = 0.0;
    r -= c1[0] * (double)a1;
    r -= c1[1] * (double)o1.carried;
    r -= c1[2] * (double)short1;
    r -= c1[3] * (double)o1.wasted;
    r += c1[4] * (double)o1.issued;
    r -= c2[0] * (double)a2;
    r -= c2[1] * (double)o2.carried;
    r -= c2[2] * (double)short2;
    r -= c2[3] * (double)o2.wasted;
    r += c2[4] * (double)o2.issued;
    out->s_next = o1.s_next + S1 * o2.s_next;
    out->reward = r;
    out->demand = d1 + d2;
    out->issued = o1.issued + o2.issued;
    out->wasted = o1.wasted + o2.wasted;
    out->carried = o1.carried + o2.carried;
    out->arrived = o1.arrived + o2.arrived;
    out->shortage = short1 + short2;
    out->unmet1 = unmet1;
    out->demand_k[0] = d1;
    out->demand_k[1] = d2;
    out->issued_k[0] = o1.issued;
    out->issued_k[1] = o2.issued;
    out->wasted_k[0] = o1.wasted;
    out->wasted_k[1] = o2.wasted;
    out->carried_k[0] = o1.carried;
    out->carried_k[1] = o2.carried;
    out->arrived_k[0] = o1.arrived;
    out->arrived_k[1] = o2.arrived;
    out->sub_served = sub_served;
    return 0;
}

/* Units available to product k this period for action a_k: the stock slots plus
 * the arrival (P_1 when L >= 2, else the order itself). */
static int units_available(const orc_problem *P, int k, long long sk, int ak) {
    prod_out o;
    product_step(P->m[k], P->L[k], P->Q[k], P->issuing, sk, ak, 0, &o);
    return o.total;
}

/* Scenario B appendix, issued-units outcome set.  Read with product 1 = B and
 * product 2 = A:
 *   P(h1, h2) = 0                                   h1 > I1 or h2 > I2
 *             = P(D1 = h1) P(D2 = h2)               h1 < I1, h2 < I2
 *             = P(D1 = h1) P(D2 >= I2)              h1 < I1, h2 = I2
 *             = P(Dz = h2) P(D1 >= I1)              h1 = I1, h2 < I2
 *             = (1 - sum_{d < I2} P(Dz = d)) P(D1 >= I1)   h1 = I1, h2 = I2
 * with Dz = D2 + Du the product-2 demand including substitutes, and Du the
 * substituting part of the product-1 shortfall c = D1 - I1 given D1 >= I1:
 *   P(Du = x) = sum_{c >= x} P(D1 = c + I1) Bin(x; c, rho) / P(D1 >= I1).
 * The printed series for Du omits the division by P(D1 >= I1); without it the
 * five cases would not sum to one, so it is read as the conditional law. */
int orc_issued_pmf(const orc_problem *P, long long s, int a, double *out, int T_out[2]) {
    if (!valid(P) || P->n_products != 2) return 1;
    ensure_binom(P);
    long long S1 = product_states(P, 0);
    long long s1 = s % S1, s2 = s / S1;
    int A2 = P->Q[1] + 1;
    int a1 = a / A2, a2 = a % A2;
    const int I1 = units_available(P, 0, s1, a1);
    const int I2 = units_available(P, 1, s2, a2);
    const double *p1 = P->pmf[0], *p2 = P->pmf[1];
    const int D1 = P->dmax[0], D2 = P->dmax[1];
#define PD1(d) (((d) >= 0 && (d) <= D1) ? p1[(d)] : 0.0)
#define PD2(d) (((d) >= 0 && (d) <= D2) ? p2[(d)] : 0.0)
    double ge1 = 0.0, ge2 = 0.0;   /* P(D1 >= I1), P(D2 >= I2) */
    for (int d = I1; d <= D1; ++d) ge1 += PD1(d);
    for (int d = I2; d <= D2; ++d) ge2 += PD2(d);
    /* P(Du = x | D1 >= I1) for x = 0..D1 - I1, then P(Dz = z) for z < I2 */
    int nu = D1 - I1 + 1;
    if (nu < 1) nu = 1;
    double *du = (double *)calloc((size_t)nu, sizeof(double));
    double *dz = (double *)calloc((size_t)(I2 + 1), sizeof(double));
    if (!du || !dz) { free(du); free(dz); return 2; }
    if (ge1 > 0.0) {
        for (int x = 0; x < nu; ++x) {
            double acc = 0.0;
            for (int c = x; c + I1 <= D1; ++c) acc += PD1(c + I1) * binom_pmf(c, x, P->rho);
            du[x] = acc / ge1;
        }
    }
    for (int z = 0; z <= I2; ++z) {
        double acc = 0.0;
        for (int k = 0; k <= z; ++k) acc += PD2(k) * ((z - k) < nu ? du[z - k] : 0.0);
        dz[z] = acc;
    }
    for (int h1 = 0; h1 <= I1; ++h1)
        for (int h2 = 0; h2 <= I2; ++h2) {
            double v;
            if (h1 < I1 && h2 < I2) {
                v = PD1(h1) * PD2(h2);
            } else if (h1 < I1) {
                v = PD1(h1) * ge2;
            } else if (h2 < I2) {
                v = dz[h2] * ge1;
            } else {
                double below = 0.0;
                for (int d = 0; d < I2; ++d) below += dz[d];
                v = (1.0 - below) * ge1;
            }
            out[(long long)h1 * (I2 + 1) + h2] = v;
        }
#undef PD1
#undef PD2
    free(du);
    free(dz);
    if (T_out) { T_out[0] = I1; T_out[1] = I2; }
    return 0;
}

/* Q(s, a) = sum_omega P(omega) [r_omega + gamma V(s'_omega)], omega ascending. */
static double q_value(const orc_problem *P, const double *V, long long s, int a) {
    double q = 0.0;
    orc_step st;
    if (P->n_products == 1) {
        for (int d = 0; d <= P->dmax[0]; ++d) {
            double p = P->pmf[0][d];
            orc_transition(P, s, a, d, 0, 0, &st);
            q += p * (st.reward + P->gamma * V[st.s_next]);
        }
        return q;
    }
    for (int d1 = 0; d1 <= P->dmax[0]; ++d1) {
        for (int d2 = 0; d2 <= P->dmax[1]; ++d2) {
            double p12 = P->pmf[0][d1] * P->pmf[1][d2];
            orc_transition(P, s, a, d1, d2, 0, &st);
            int n = st.unmet1;
            for (int u = 0; u <= n; ++u) {
                double p = p12 * binom_pmf(n, u, P->rho);
                orc_transition(P, s, a, d1, d2, u, &st);
                q += p * (st.reward + P->gamma * V[st.s_next]);
            }
        }
    }
    return q;
}

int orc_qvalues(const orc_problem *P, const double *V, long long s, double *q) {
    ensure_binom(P);
    int A = orc_num_actions(P);
    for (int a = 0; a < A; ++a) q[a] = q_value(P, V, s, a);
    return 0;
}

static void backup_one(const orc_problem *P, const double *V, long long s, double *v, int *pol) {
    int A = orc_num_actions(P);
    double best = -INFINITY;
    int arg = 0;
    for (int a = 0; a < A; ++a) {
        double q = q_value(P, V, s, a);
        if (q > best) { best = q; arg = a; }
    }
    *v = best;
    *pol = arg;
}

static int valid(const orc_problem *P) {
    if (P->n_products != 1 && P->n_products != 2) return 0;
    for (int k = 0; k < P->n_products; ++k) {
        if (P->m[k] < 1 || P->L[k] < 1 || P->Q[k] < 0 || P->dmax[k] < 0) return 0;
        if ((P->m[k] - 1) + (P->L[k] - 1) > MAXDIG) return 0;
    }
    return 1;
}

int orc_vi_solve(const orc_problem *P, double tol, int stop_rule, int max_iters,
                 double *V, uint8_t *policy, int *iters, double *crit_out,
                 double *dmax_out, double *dmin_out, int nthreads) {
    if (!valid(P)) return 1;
    ensure_binom(P);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    long long S = orc_num_states(P);
    double *cur = V;
    double *nxt = (double *)malloc(sizeof(double) * (size_t)S);
    if (!nxt) return 2;
    int converged = 0, i = 0;
    double crit = INFINITY, dmx = 0.0, dmn = 0.0;
    while (i < max_iters) {
        ++i;
#pragma omp parallel for schedule(static)
        for (long long s = 0; s < S; ++s) {
            int pol;
            backup_one(P, cur, s, &nxt[s], &pol);
        }
        dmx = -INFINITY;
        dmn = INFINITY;
        for (long long s = 0; s < S; ++s) {
            double d = nxt[s] - cur[s];
            if (d > dmx) dmx = d;
            if (d < dmn) dmn = d;
        }
        double *t = cur; cur = nxt; nxt = t;
        crit = (stop_rule == 1) ? fmax(fabs(dmx), fabs(dmn)) : (dmx - dmn);
        if (crit < tol) { converged = 1; break; }
    }
    if (cur != V) {
        memcpy(V, cur, sizeof(double) * (size_t)S);
        nxt = cur;
    }
    if (policy) {
#pragma omp parallel for schedule(static)
        for (long long s = 0; s < S; ++s) {
            double v;
            int pol;
            backup_one(P, V, s, &v, &pol);
            policy[s] = (uint8_t)pol;
        }
    }
    free(nxt);
    if (iters) *iters = i;
    if (crit_out) *crit_out = crit;
    if (dmax_out) *dmax_out = dmx;
    if (dmin_out) *dmin_out = dmn;
    return converged ? 0 : 3;
}

int orc_backup_states(const orc_problem *P, const double *V, const long long *states,
                      long long n, double *v_out, int *pol_out, double *q_out, int nthreads) {
    if (!valid(P)) return 1;
    ensure_binom(P);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    int A = orc_num_actions(P);
#pragma omp parallel for schedule(dynamic, 16)
    for (long long i = 0; i < n; ++i) {
        double v;
        int pol;
        backup_one(P, V, states[i], &v, &pol);
        if (v_out) v_out[i] = v;
        if (pol_out) pol_out[i] = pol;
        if (q_out) orc_qvalues(P, V, states[i], q_out + i * A);
    }
    return 0;
}

int orc_policy_eval(const orc_problem *P, const uint8_t *policy, double tol, int max_iters,
                    double *V, int *iters, int nthreads) {
    if (!valid(P)) return 1;
    ensure_binom(P);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    long long S = orc_num_states(P);
    double *nxt = (double *)malloc(sizeof(double) * (size_t)S);
    double *cur = V;
    if (!nxt) return 2;
    int i = 0, converged = 0;
    while (i < max_iters) {
        ++i;
#pragma omp parallel for schedule(static)
        for (long long s = 0; s < S; ++s) nxt[s] = q_value(P, cur, s, policy[s]);
        double sup = 0.0;
        for (long long s = 0; s < S; ++s) sup = fmax(sup, fabs(nxt[s] - cur[s]));
        double *t = cur; cur = nxt; nxt = t;
        if (sup < tol) { converged = 1; break; }
    }
    if (cur != V) {
        memcpy(V, cur, sizeof(double) * (size_t)S);
        nxt = cur;
    }
    free(nxt);
    if (iters) *iters = i;
    return converged ? 0 : 3;
}

/* ---------------------------------------------------------------------------
 * Philox4x32-10, from the description in Salmon et al. (SC'11): each round
 * multiplies words 0 and 2 by the constants 0xD2511F53 and 0xCD9E8D57 into
 * 64-bit products, and the new block is
 *   (hi(M1*x2) ^ x1 ^ k0, lo(M1*x2), hi(M0*x0) ^ x3 ^ k1, lo(M0*x0));
 * the key is bumped by the Weyl constants (0x9E3779B9, 0xBB67AE85) between
 * rounds.
 * ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Demand from one 32-bit uniform word: the smallest d with w < thr[d], where
 * thr[d] = floor(2^32 * CDF(d)) with CDF summed in ascending order in FP64,
 * clipped to 2^32, and thr[dmax] = 2^32. */
static void make_thresholds(const double *pmf, int dmax, uint64_t *thr) {
    double cdf = 0.0;
    for (int d = 0; d <= dmax; ++d) {
        cdf += pmf[d];
        double t = floor(cdf * 4294967296.0);
        if (t > 4294967296.0) t = 4294967296.0;
        if (t < 0.0) t = 0.0;
        thr[d] = (uint64_t)t;
    }
    thr[dmax] = 4294967296ull;
}

static int draw_demand(uint32_t w, const uint64_t *thr, int dmax) {
    int d = 0;
    while (d < dmax && (uint64_t)w >= thr[d]) ++d;
    return d;
}

static int popcount32(uint32_t x) {
    int c = 0;
    while (x) { c += (int)(x & 1u); x >>= 1; }
    return c;
}

/* per-product KPI sums of one rollout */
typedef struct {
    double dem[2], served[2], was[2], arr[2], car[2];
} kpi_sums;

static void kpi_sums_finish(const kpi_sums *k, int horizon, double *out6) {
    for (int j = 0; j < 2; ++j) {
        out6[3 * j + 0] = k->dem[j] > 0.0 ? 100.0 * k->served[j] / k->dem[j] : 100.0;
        out6[3 * j + 1] = k->arr[j] > 0.0 ? 100.0 * k->was[j] / k->arr[j] : 0.0;
        out6[3 * j + 2] = horizon > 0 ? k->car[j] / (double)horizon : 0.0;
    }
}

/* the substituting customers among n: popcount of the low n bits of the 64-bit
 * word (word 3, word 2) -- bits 0..31 from word 2, bits 32..63 from word 3 */
static int substitutes(uint32_t w2, uint32_t w3, int n) {
    const int lo = n < 32 ? n : 32;
    const int hi = n > 64 ? 32 : (n > 32 ? n - 32 : 0);
    const uint32_t mlo = (lo >= 32) ? 0xffffffffu : ((1u << lo) - 1u);
    const uint32_t mhi = (hi >= 32) ? 0xffffffffu : ((1u << hi) - 1u);
    return popcount32(w2 & mlo) + popcount32(w3 & mhi);
}

int orc_simulate(const orc_problem *P, const uint8_t *policy, int n_rollouts, int horizon,
                 int warmup, uint64_t seed, double *returns, double *kpis, int32_t *traj,
                 int32_t *demand_out) {
    return orc_simulate_ex(P, policy, n_rollouts, horizon, warmup, seed, returns, kpis, NULL, traj,
                           demand_out);
}

int orc_simulate_ex(const orc_problem *P, const uint8_t *policy, int n_rollouts, int horizon,
                    int warmup, uint64_t seed, double *returns, double *kpis, double *kpis_prod,
                    int32_t *traj, int32_t *demand_out) {
    if (!valid(P)) return 1;
    if (P->n_products == 2 && P->rho != 0.5) return 1;
    uint64_t thr0[512], thr1[512];
    if (P->dmax[0] >= 512 || (P->n_products == 2 && P->dmax[1] >= 512)) return 1;
    make_thresholds(P->pmf[0], P->dmax[0], thr0);
    if (P->n_products == 2) make_thresholds(P->pmf[1], P->dmax[1], thr1);
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    for (int r = 0; r < n_rollouts; ++r) {
        long long s = 0;
        double ret = 0.0, disc = 1.0;
        double dem = 0.0, iss = 0.0, was = 0.0, arr = 0.0, car = 0.0;
        kpi_sums ks;
        memset(&ks, 0, sizeof(ks));
        for (int t = 0; t < warmup + horizon; ++t) {
            uint32_t ctr[4] = {(uint32_t)t, (uint32_t)r, 0u, 0u}, w[4];
            orc_philox4x32_10(ctr, key, w);
            int d1 = draw_demand(w[0], thr0, P->dmax[0]);
            int d2 = 0, u = 0;
            int a = policy[s];
            orc_step st;
            if (P->n_products == 2) {
                d2 = draw_demand(w[1], thr1, P->dmax[1]);
                orc_transition(P, s, a, d1, d2, 0, &st);
                u = substitutes(w[2], w[3], st.unmet1);
            }
            orc_transition(P, s, a, d1, d2, u, &st);
            if (t >= warmup) {
                int tt = t - warmup;
                if (traj) traj[(long long)r * horizon + tt] = (int32_t)s;
                if (demand_out) demand_out[(long long)r * horizon + tt] = d1;
                ret += disc * st.reward;
                disc *= P->gamma;
                dem += st.demand;
                iss += st.issued;
                was += st.wasted;
                arr += st.arrived;
                car += st.carried;
                ks.dem[0] += st.demand_k[0];
                ks.dem[1] += st.demand_k[1];
                ks.served[0] += st.issued_k[0] + (double)st.sub_served;
                ks.served[1] += st.issued_k[1] - (double)st.sub_served;
                for (int j = 0; j < 2; ++j) {
                    ks.was[j] += st.wasted_k[j];
                    ks.arr[j] += st.arrived_k[j];
                    ks.car[j] += st.carried_k[j];
                }
            }
            s = st.s_next;
        }
        returns[r] = ret;
        if (kpis) {
            kpis[3 * r + 0] = dem > 0.0 ? 100.0 * iss / dem : 100.0;
            kpis[3 * r + 1] = arr > 0.0 ? 100.0 * was / arr : 0.0;
            kpis[3 * r + 2] = horizon > 0 ? car / (double)horizon : 0.0;
        }
        if (kpis_prod) kpi_sums_finish(&ks, horizon, kpis_prod + 6 * (long long)r);
    }
    return 0;
}

/* ---------------------------------------------------------------------------
 * Modified base-stock heuristic on plain stock vectors.  One product, one
 * period: Y_1..Y_{m-1} = X_1..X_{m-1} (Y_1 expires), Y_m = the arrival; z units
 * are issued FIFO (oldest first) or LIFO (freshest first), the rest of Y_1 is
 * wasted and the others age by one period (the issuing equations of Scenario A
 * and Scenario B, applied slot by slot).
 * ------------------------------------------------------------------------- */
typedef struct {
    int X[MAXDIG + 2];      /* X[1..m-1] */
    int Pp[MAXDIG + 2];     /* P[1..L-1] */
} stock_vec;

static void vec_period(const orc_problem *P, int k, stock_vec *v, int order, int z, prod_out *o) {
    const int m = P->m[k], L = P->L[k];
    int Y[MAXDIG + 2];
    for (int j = 1; j <= m - 1; ++j) Y[j] = v->X[j];
    Y[m] = (L >= 2) ? v->Pp[1] : order;
    int T = 0;
    for (int j = 1; j <= m; ++j) T += Y[j];
    int left = z;   /* demand not yet met */
    int rem[MAXDIG + 2] = {0};
    for (int j = 1; j <= m; ++j) rem[j] = Y[j];
    if (P->issuing == 0) {
        for (int j = 1; j <= m && left > 0; ++j) {
            int take = imin(rem[j], left);
            rem[j] -= take;
            left -= take;
        }
    } else {
        for (int j = m; j >= 1 && left > 0; --j) {
            int take = imin(rem[j], left);
            rem[j] -= take;
            left -= take;
        }
    }
    o->total = T;
    o->issued = imin(z, T);
    o->wasted = rem[1];
    o->shortage = ipos(z - T);
    o->arrived = Y[m];
    int car = 0;
    for (int j = 1; j <= m - 1; ++j) {
        v->X[j] = rem[j + 1];
        car += rem[j + 1];
    }
    o->carried = car;
    for (int j = 1; j <= L - 2; ++j) v->Pp[j] = v->Pp[j + 1];
    if (L >= 2) v->Pp[L - 1] = order;
    o->s_next = 0;
}

int orc_mbs_simulate(const orc_problem *P, const int S[2], const int mu[2], int cap, int n_rollouts,
                     int horizon, int warmup, uint64_t seed, double *returns, double *kpis_prod) {
    if (!valid(P) || !S || !mu) return 1;
    if (P->n_products == 2 && P->rho != 0.5) return 1;
    const int np = P->n_products;
    uint64_t thr[2][512];
    for (int k = 0; k < np; ++k) {
        if (P->dmax[k] >= 512) return 1;
        make_thresholds(P->pmf[k], P->dmax[k], thr[k]);
    }
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    for (int r = 0; r < n_rollouts; ++r) {
        stock_vec v[2];
        memset(v, 0, sizeof(v));
        double ret = 0.0, disc = 1.0;
        kpi_sums ks;
        memset(&ks, 0, sizeof(ks));
        for (int t = 0; t < warmup + horizon; ++t) {
            uint32_t ctr[4] = {(uint32_t)t, (uint32_t)r, 0u, 0u}, w[4];
            orc_philox4x32_10(ctr, key, w);
            int order[2] = {0, 0};
            for (int k = 0; k < np; ++k) {
                int onhand = 0;
                for (int j = 1; j <= P->m[k] - 1; ++j) onhand += v[k].X[j];
                if (P->L[k] >= 2) onhand += v[k].Pp[1];
                int expiring = (P->m[k] >= 2) ? v[k].X[1] : ((P->L[k] >= 2) ? v[k].Pp[1] : 0);
                int q = S[k] - onhand + ipos(expiring - mu[k]);
                q = ipos(q);
                if (cap && q > P->Q[k]) q = P->Q[k];
                order[k] = q;
            }
            const int d1 = draw_demand(w[0], thr[0], P->dmax[0]);
            const int d2 = (np == 2) ? draw_demand(w[1], thr[1], P->dmax[1]) : 0;
            prod_out o1, o2;
            vec_period(P, 0, &v[0], order[0], d1, &o1);
            double rew = 0.0;
            int sub = 0, short1 = o1.shortage, short2 = 0;
            if (np == 2) {
                const int u = substitutes(w[2], w[3], o1.shortage);
                vec_period(P, 1, &v[1], order[1], d2 + u, &o2);
                const int own2 = imin(d2, o2.total);
                sub = o2.issued - own2;
                short1 = o1.shortage - sub;
                short2 = ipos(d2 - o2.total);
            }
            const double *c1 = P->cost[0];
            rew -= c1[0] * (double)order[0];
            rew -= c1[1] * (double)o1.carried;
            rew -= c1[2] * (double)short1;
            rew -= c1[3] * (double)o1.wasted;
            rew += c1[4] * (double)o1.issued;
            if (np == 2) {
                const double *c2 = P->cost[1];
                rew -= c2[0] * (double)order[1];
                rew -= c2[1] * (double)o2.carried;
                rew -= c2[2] * (double)short2;
                rew -= c2[3] * (double)o2.wasted;
                rew += c2[4] * (double)o2.issued;
            }
            if (t >= warmup) {
                ret += disc * rew;
                disc *= P->gamma;
                ks.dem[0] += d1;
                ks.served[0] += o1.issued + sub;
                ks.was[0] += o1.wasted;
                ks.arr[0] += o1.arrived;
                ks.car[0] += o1.carried;
                if (np == 2) {
                    ks.dem[1] += d2;
                    ks.served[1] += o2.issued - sub;
                    ks.was[1] += o2.wasted;
                    ks.arr[1] += o2.arrived;
                    ks.car[1] += o2.carried;
                }
            }
        }
        returns[r] = ret;
        if (kpis_prod) kpi_sums_finish(&ks, horizon, kpis_prod + 6 * (long long)r);
    }
    return 0;
}

/* Base-stock heuristic (Methods, Scenario A): A = [S - I]^+ with I the total
 * stock on hand and in transit, i.e. the sum of all digits of the state. */
int orc_basestock_policy(const orc_problem *P, int S, uint8_t *policy) {
    if (!valid(P) || P->n_products != 1 || !policy || S < 0) return 1;
    const long long n = orc_num_states(P);
    const int G = P->Q[0] + 1;
    const int K = (P->m[0] - 1) + (P->L[0] - 1);
    for (long long s = 0; s < n; ++s) {
        long long rem = s;
        int stock = 0;
        for (int k = 0; k < K; ++k) {
            stock += (int)(rem % G);
            rem /= G;
        }
        int a = S - stock;
        if (a < 0) a = 0;
        if (a > P->Q[0]) a = P->Q[0];
        policy[s] = (uint8_t)a;
    }
    return 0;
}
