/*
 * oracle_pc.c -- plain FP64 CPU value iteration and rollouts for the paper's
 * Scenario C (periodic demand and uncertain useful life on arrival; Scenario C
 * appendix).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU legs, never by the product path.  Nothing here is shared
 * with the CUDA library.
 *
 * Everything is evaluated per outcome, the slow obvious way:
 *   - state (tau, X_1..X_{m-1}): tau the weekday, X_j the units with j days of
 *     useful life left (X_1 expires at the end of today), each 0..A_max;
 *   - outcome (d, y_1..y_m): the day's demand (truncated negative binomial of
 *     weekday tau, Eq. mirjalili:demand) and the units received with k days of
 *     life left (multinomial over the a units ordered, Eq.
 *     mirjalili:ageonarrival, with log(p_k / p_1) = c0_k + c1_k a);
 *   - units in excess of A_max for an age are refused at delivery:
 *     Z_j = min(X_j + y_j, A_max) for j < m, Z_m = y_m;
 *   - issuing oldest unit first, next state and reward per the Scenario C
 *     appendix (Eq. mirjalili:state_transition and the reward equation);
 *   - Q(s, a) = sum_y P(y | a) sum_d P(d | tau) [r + gamma V(s')], y in the
 *     order of orc_pc_next_profile, d ascending;
 *   - stopping: the periodic test of Su and Deininger (Scenario C appendix):
 *     for i >= 7, Delta_i(s) = sum_{j=0}^{6} gamma^-(i-j-1) (V_{i-j}(s) -
 *     V_{i-j-1}(s)); stop when max Delta - min Delta <= 2 eps min(|max|, |min|).
 * Build with -ffp-contract=off so that no multiply-add is fused.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PC_MAXM 8

static int pc_valid(const orc_periodic *P) {
    if (!P || P->m < 2 || P->m > PC_MAXM || P->Q < 0 || P->dmax < 0 || !P->pmf) return 0;
    if (!(P->gamma > 0.0 && P->gamma < 1.0)) return 0;
    return 1;
}

long long orc_pc_num_states(const orc_periodic *P) {
    long long n = 7;
    for (int j = 1; j < P->m; ++j) n *= (P->Q + 1);
    return n;
}

/* multinomial parameters p_1(a)..p_m(a) from the affine logits */
void orc_pc_arrival_params(const orc_periodic *P, int a, double *p) {
    double z = 1.0;
    double e[PC_MAXM + 1];
    e[1] = 1.0;
    for (int k = 2; k <= P->m; ++k) {
        e[k] = exp(P->c0[k] + P->c1[k] * (double)a);
        z += e[k];
    }
    for (int k = 1; k <= P->m; ++k) p[k] = e[k] / z;
}

/* P(Y = y | A = a): a! / (y_1! ... y_m!) prod p_k(a)^y_k when sum y = a, else 0.
 * The multinomial coefficient is built as a product of binomial coefficients. */
double orc_pc_arrival_prob(const orc_periodic *P, int a, const int *y) {
    int sum = 0;
    for (int k = 1; k <= P->m; ++k) {
        if (y[k] < 0) return 0.0;
        sum += y[k];
    }
    if (sum != a) return 0.0;
    double p[PC_MAXM + 1];
    orc_pc_arrival_params(P, a, p);
    double coef = 1.0;
    int left = a;
    for (int k = 1; k <= P->m; ++k) {
        /* C(left, y_k), exact for left <= 60 */
        double c = 1.0;
        for (int i = 1; i <= y[k]; ++i) c = c * (double)(left - y[k] + i) / (double)i;
        coef *= c;
        left -= y[k];
    }
    double pr = coef;
    for (int k = 1; k <= P->m; ++k) pr *= pow(p[k], (double)y[k]);
    return pr;
}

/* Advance y[1..m] to the next composition of a (y_1 varies fastest after the
 * others are fixed: the enumeration runs y_m = 0..a outermost, then y_{m-1},
 * ..., with y_1 = the rest).  Start with y_m = ... = y_2 = 0, y_1 = a.
 * Returns 0 when the enumeration is exhausted. */
int orc_pc_next_profile(int m, int a, int *y) {
    /* find the lowest k >= 2 that can be increased: raising y_k takes one unit
       from the rest, y_1 = a - sum_{k>=2} y_k */
    for (int k = 2; k <= m; ++k) {
        int higher = 0;
        for (int j = k + 1; j <= m; ++j) higher += y[j];
        if (higher + y[k] < a) {
            y[k] += 1;
            for (int j = 2; j < k; ++j) y[j] = 0;
            int rest = 0;
            for (int j = 2; j <= m; ++j) rest += y[j];
            y[1] = a - rest;
            return 1;
        }
    }
    return 0;
}

static void decode(const orc_periodic *P, long long s, int *tau, int *X) {
    const int G = P->Q + 1;
    long long rem = s;
    for (int j = 1; j <= P->m - 1; ++j) {
        X[j] = (int)(rem % G);
        rem /= G;
    }
    *tau = (int)rem;
}

static long long encode(const orc_periodic *P, int tau, const int *X) {
    const int G = P->Q + 1;
    long long s = tau;
    for (int j = P->m - 1; j >= 1; --j) s = s * G + X[j];
    return s;
}

int orc_pc_transition(const orc_periodic *P, long long s, int a, int d, const int *y, orc_pc_step *out) {
    if (!pc_valid(P) || a < 0 || a > P->Q || d < 0 || d > P->dmax) return 1;
    const int m = P->m, A = P->Q;
    int tau, X[PC_MAXM + 1];
    decode(P, s, &tau, X);
    int sum = 0;
    for (int k = 1; k <= m; ++k) sum += y[k];
    if (sum != a) return 1;
    /* units in stock after delivery, with the per-age capacity */
    int Z[PC_MAXM + 1];
    int accepted = 0;
    for (int j = 1; j <= m - 1; ++j) {
        const int t = X[j] + y[j];
        Z[j] = t < A ? t : A;
        accepted += Z[j] - X[j];
    }
    Z[m] = y[m];
    accepted += y[m];
    int T = 0;
    for (int j = 1; j <= m; ++j) T += Z[j];
    /* oldest unit first: X'_j = [Z_{j+1} - [d - sum_{k<=j} Z_k]^+]^+ */
    int Xn[PC_MAXM + 1];
    int cum = 0;
    for (int j = 1; j <= m - 1; ++j) {
        cum += Z[j];
        int reach = d - cum;
        if (reach < 0) reach = 0;
        int v = Z[j + 1] - reach;
        Xn[j] = v > 0 ? v : 0;
    }
    const int left = T - d > 0 ? T - d : 0;
    const int shortage = d - T > 0 ? d - T : 0;
    const int wasted = Z[1] - d > 0 ? Z[1] - d : 0;
    double r = 0.0;
    if (a > 0) r -= P->cost[0];
    r -= P->cost[1] * (double)left;
    r -= P->cost[2] * (double)shortage;
    r -= P->cost[3] * (double)wasted;
    out->s_next = encode(P, (tau + 1) % 7, Xn);
    out->reward = r;
    out->demand = d;
    out->issued = d < T ? d : T;
    out->wasted = wasted;
    out->held = left;
    out->accepted = accepted;
    out->refused = a - accepted;
    return 0;
}

static double pc_q(const orc_periodic *P, const double *V, long long s, int a) {
    const int m = P->m;
    int tau, X[PC_MAXM + 1];
    decode(P, s, &tau, X);
    const double *pd = P->pmf + (long long)tau * (P->dmax + 1);
    int y[PC_MAXM + 1];
    for (int k = 1; k <= m; ++k) y[k] = 0;
    y[1] = a;
    double q = 0.0;
    orc_pc_step st;
    do {
        const double py = orc_pc_arrival_prob(P, a, y);
        for (int d = 0; d <= P->dmax; ++d) {
            orc_pc_transition(P, s, a, d, y, &st);
            q += py * pd[d] * (st.reward + P->gamma * V[st.s_next]);
        }
    } while (orc_pc_next_profile(m, a, y));
    return q;
}

int orc_pc_qvalues(const orc_periodic *P, const double *V, long long s, double *q) {
    if (!pc_valid(P)) return 1;
    for (int a = 0; a <= P->Q; ++a) q[a] = pc_q(P, V, s, a);
    return 0;
}

static void pc_backup_one(const orc_periodic *P, const double *V, long long s, double *v, int *pol) {
    double best = -INFINITY;
    int arg = 0;
    for (int a = 0; a <= P->Q; ++a) {
        const double q = pc_q(P, V, s, a);
        if (q > best) { best = q; arg = a; }
    }
    *v = best;
    *pol = arg;
}

int orc_pc_backup_states(const orc_periodic *P, const double *V, const long long *states, long long n,
                         double *v_out, int *pol_out, int nthreads) {
    if (!pc_valid(P)) return 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 4)
    for (long long i = 0; i < n; ++i) {
        double v;
        int pol;
        pc_backup_one(P, V, states[i], &v, &pol);
        if (v_out) v_out[i] = v;
        if (pol_out) pol_out[i] = pol;
    }
    return 0;
}

int orc_pc_vi_solve(const orc_periodic *P, double eps, int stop_rule, int max_iters, double *V, uint8_t *policy,
                    int *iters, double *crit_out, double *dmax_out, double *dmin_out, int nthreads) {
    if (!pc_valid(P) || stop_rule < 0 || stop_rule > 2) return 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    const long long S = orc_pc_num_states(P);
    /* hist[k] = V_{i-k}, k = 0..7 (the periodic test needs the last eight) */
    double *hist[8];
    for (int k = 0; k < 8; ++k) {
        hist[k] = (double *)malloc(sizeof(double) * (size_t)S);
        if (!hist[k]) {
            for (int j = 0; j < k; ++j) free(hist[j]);
            return 2;
        }
    }
    memcpy(hist[0], V, sizeof(double) * (size_t)S);
    int i = 0, converged = 0;
    double crit = INFINITY, dmx = 0.0, dmn = 0.0;
    while (i < max_iters) {
        ++i;
        /* rotate: the oldest buffer receives V_i */
        double *nw = hist[7];
        for (int k = 7; k > 0; --k) hist[k] = hist[k - 1];
        hist[0] = nw;
#pragma omp parallel for schedule(dynamic, 4)
        for (long long s = 0; s < S; ++s) {
            int pol;
            pc_backup_one(P, hist[1], s, &hist[0][s], &pol);
        }
        if (stop_rule == 2) {
            if (i < 7) continue;
            dmx = -INFINITY;
            dmn = INFINITY;
            for (long long s = 0; s < S; ++s) {
                double delta = 0.0;
                for (int j = 0; j <= 6; ++j)
                    delta += (hist[j][s] - hist[j + 1][s]) / pow(P->gamma, (double)(i - j - 1));
                if (delta > dmx) dmx = delta;
                if (delta < dmn) dmn = delta;
            }
            crit = (dmx - dmn) / fmin(fabs(dmx), fabs(dmn));
            if (dmx - dmn <= 2.0 * eps * fmin(fabs(dmx), fabs(dmn))) { converged = 1; break; }
        } else {
            dmx = -INFINITY;
            dmn = INFINITY;
            for (long long s = 0; s < S; ++s) {
                const double dl = hist[0][s] - hist[1][s];
                if (dl > dmx) dmx = dl;
                if (dl < dmn) dmn = dl;
            }
            crit = (stop_rule == 1) ? fmax(fabs(dmx), fabs(dmn)) : (dmx - dmn);
            if (crit < eps) { converged = 1; break; }
        }
    }
    memcpy(V, hist[0], sizeof(double) * (size_t)S);
    if (policy) {
#pragma omp parallel for schedule(dynamic, 4)
        for (long long s = 0; s < S; ++s) {
            double v;
            int pol;
            pc_backup_one(P, V, s, &v, &pol);
            policy[s] = (uint8_t)pol;
        }
    }
    for (int k = 0; k < 8; ++k) free(hist[k]);
    if (iters) *iters = i;
    if (crit_out) *crit_out = crit;
    if (dmax_out) *dmax_out = dmx;
    if (dmin_out) *dmin_out = dmn;
    return converged ? 0 : 3;
}

/* thresholds floor(2^32 CDF) of a pmf summed in ascending order, last = 2^32 */
static void pc_thresholds(const double *pmf, int n, uint64_t *thr) {
    double cdf = 0.0;
    for (int i = 0; i < n; ++i) {
        cdf += pmf[i];
        double t = floor(cdf * 4294967296.0);
        if (t > 4294967296.0) t = 4294967296.0;
        if (t < 0.0) t = 0.0;
        thr[i] = (uint64_t)t;
    }
    thr[n - 1] = 4294967296ull;
}

static int pc_draw(uint32_t w, const uint64_t *thr, int n) {
    int i = 0;
    while (i < n - 1 && (uint64_t)w >= thr[i]) ++i;
    return i;
}

int orc_pc_simulate(const orc_periodic *P, const uint8_t *policy, int n_rollouts, int horizon, int warmup,
                    uint64_t seed, double *returns, double *kpis, int32_t *traj) {
    if (!pc_valid(P) || P->dmax >= 512 || P->Q > 255) return 1;
    const int m = P->m;
    uint64_t thr_d[7][512];
    for (int t = 0; t < 7; ++t) pc_thresholds(P->pmf + (long long)t * (P->dmax + 1), P->dmax + 1, thr_d[t]);
    /* age-class thresholds per order size: class k-1 (k = 1..m) of one unit */
    uint64_t *thr_y = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(P->Q + 1) * m);
    if (!thr_y) return 2;
    for (int a = 0; a <= P->Q; ++a) {
        double p[PC_MAXM + 1];
        orc_pc_arrival_params(P, a, p);
        pc_thresholds(p + 1, m, thr_y + (size_t)a * m);
    }
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    for (int r = 0; r < n_rollouts; ++r) {
        long long s = 0;
        double ret = 0.0, disc = 1.0;
        double dem = 0.0, iss = 0.0, was = 0.0, acc = 0.0, held = 0.0;
        for (int t = 0; t < warmup + horizon; ++t) {
            uint32_t ctr[4] = {(uint32_t)t, (uint32_t)r, 0u, 0u}, w[4];
            orc_philox4x32_10(ctr, key, w);
            const int tau = (int)(s / (orc_pc_num_states(P) / 7));
            const int d = pc_draw(w[0], thr_d[tau], P->dmax + 1);
            const int a = policy[s];
            int y[PC_MAXM + 1];
            for (int k = 1; k <= m; ++k) y[k] = 0;
            for (int u = 0; u < a; ++u) {
                uint32_t c2[4] = {(uint32_t)t, (uint32_t)r, (uint32_t)(1 + u / 4), 0u}, wu[4];
                orc_philox4x32_10(c2, key, wu);
                y[1 + pc_draw(wu[u % 4], thr_y + (size_t)a * m, m)] += 1;
            }
            orc_pc_step st;
            orc_pc_transition(P, s, a, d, y, &st);
            if (t >= warmup) {
                if (traj) traj[(long long)r * horizon + (t - warmup)] = (int32_t)s;
                ret += disc * st.reward;
                disc *= P->gamma;
                dem += st.demand;
                iss += st.issued;
                was += st.wasted;
                acc += st.accepted;
                held += st.held;
            }
            s = st.s_next;
        }
        returns[r] = ret;
        if (kpis) {
            kpis[3 * r + 0] = dem > 0.0 ? 100.0 * iss / dem : 100.0;
            kpis[3 * r + 1] = acc > 0.0 ? 100.0 * was / acc : 0.0;
            kpis[3 * r + 2] = horizon > 0 ? held / (double)horizon : 0.0;
        }
    }
    free(thr_y);
    return 0;
}
