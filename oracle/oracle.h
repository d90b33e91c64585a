/*
 * oracle.h -- plain FP64 CPU reference for value iteration on the perishable
 * inventory MDP of Farrington et al., "Going faster to see further" (2023).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA library under
 * paper_2303_10672_b300/ and neither includes the other.
 *
 * Model (single product; the paper's Scenario A equations, observed at the
 * decision epoch): a state holds the on-hand stock X_1..X_{m-1} by remaining
 * useful life (X_1 expires at the end of this period) and the pipeline
 * P_1..P_{L-1} (P_1 arrives before this period's demand).  The arrival
 * u = P_1 (L >= 2) or u = the action itself (L = 1) joins as the freshest slot
 * Y_m; demand is issued FIFO or LIFO (Eqs. demoor:fifo / demoor:lifo); the
 * oldest remainder is wasted; the rest ages by one period.  Reward per
 * Eq. demoor:reward plus revenue per unit issued (Scenario B reward).
 * Two products: product 1's shortfall accepts product 2 with probability rho
 * per unit (binomial, Scenario B appendix).
 *
 * State index: digit k has weight (Q+1)^k; digits 0..m-2 are X_1..X_{m-1},
 * digits m-1..m+L-3 are P_1..P_{L-1}.  Two products: s = s_1 + |S_1| * s_2.
 * Joint action a = a_1 * (Q_2 + 1) + a_2.
 */
#ifndef VI_ORACLE_H
#define VI_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int n_products;          /* 1 or 2 */
    int m[2], L[2], Q[2];    /* useful life, lead time, order cap per product */
    double cost[2][5];       /* c_o (order), c_h (holding), c_s (shortage), c_w (waste), c_r (revenue) */
    const double *pmf[2];    /* demand pmf on 0..dmax[k] */
    int dmax[2];
    double rho;              /* substitution acceptance probability (two products) */
    double gamma;            /* discount factor, 0 <= gamma <= 1 */
    int issuing;             /* 0 = FIFO, 1 = LIFO */
} orc_problem;

typedef struct {
    long long s_next;
    double reward;
    double demand;    /* total demand (both products) */
    double issued;    /* units issued (both products) */
    double wasted;    /* units expired at end of period */
    double carried;   /* units carried to the next period (on hand, not pipeline) */
    double arrived;   /* units received this period */
    double shortage;  /* demand lost after substitution */
    int unmet1;       /* product-1 shortfall before substitution (two products) */
    /* per product k (index 1 is zero for one product) */
    double demand_k[2];   /* own demand d_k */
    double issued_k[2];   /* units leaving product k's stock (product 2: own + substitutes) */
    double wasted_k[2], carried_k[2], arrived_k[2];
    int sub_served;       /* product-1 shortfall met by product 2 */
} orc_step;

long long orc_num_states(const orc_problem *P);
int orc_num_actions(const orc_problem *P);

/* One deterministic transition T(s, a, omega): omega = (d1) or (d1, d2, u). */
int orc_transition(const orc_problem *P, long long s, int a, int d1, int d2, int u, orc_step *out);

/* Q(s, a) for every action of state s from the value function V (FP64). */
int orc_qvalues(const orc_problem *P, const double *V, long long s, double *q);

/* Synchronous value iteration from V (in: V_0, out: V_i).  stop_rule 0 = span,
 * 1 = sup-norm; stops at the first i with criterion < tol or at max_iters.
 * policy (optional) gets the one-step look-ahead argmax from the returned V.
 * Returns 0 if converged, 3 if max_iters was reached, 1 on bad input. */
int orc_vi_solve(const orc_problem *P, double tol, int stop_rule, int max_iters,
                 double *V, uint8_t *policy, int *iters, double *crit_out,
                 double *dmax_out, double *dmin_out, int nthreads);

/* One Bellman update at the listed states: v_out[i] = max_a Q(states[i], a),
 * pol_out[i] = smallest argmax, q_out (optional) = n x |A| Q-values. */
int orc_backup_states(const orc_problem *P, const double *V, const long long *states,
                      long long n, double *v_out, int *pol_out, double *q_out, int nthreads);

/* Evaluate a fixed policy: V <- r_pi + gamma P_pi V from the given V until the
 * sup-norm change is < tol or max_iters.  Returns 0 / 3 like orc_vi_solve. */
int orc_policy_eval(const orc_problem *P, const uint8_t *policy, double tol, int max_iters,
                    double *V, int *iters, int nthreads);

/* Distribution of the units issued, P(h1, h2 | s, a), from the Scenario B
 * appendix's five cases (issued-units outcome set, with the substitution
 * demand D^u and the total product-2 demand D^z).  Product 1 here is the
 * paper's product B (its shortfall may take product 2), product 2 the paper's
 * product A.  out: (T1 + 1) x (T2 + 1) row-major (row h1), T_k = units of
 * product k available this period (written to T_out).  Two products only. */
int orc_issued_pmf(const orc_problem *P, long long s, int a, double *out, int T_out[2]);

/* Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Base-stock heuristic (Methods, Scenario A "Heuristic policies"): order up to
 * S counting every unit on hand and in transit, A = [S - I]^+, capped at the
 * largest order Q.  Single product; writes the action of every state. */
int orc_basestock_policy(const orc_problem *P, int S, uint8_t *policy);

/* Rollouts of a fixed policy from the all-zero state.  Period t of rollout r
 * draws Philox4x32-10(ctr = (t, r, 0, 0), key = (seed lo, seed hi)); word 0 gives
 * product-1 demand, word 1 product-2 demand, words 2 and 3 the substitution bits
 * (the popcount of the low `shortfall` bits of the 64-bit word (word 3, word 2);
 * rho must be 1/2 for two products; a shortfall above 64 uses 64 bits).  returns[r] = sum over the horizon of
 * gamma^t * reward; kpis[3r..3r+2] = service %, wastage %, mean units carried.
 * traj (optional) = n_rollouts x horizon states observed before each decision. */
int orc_simulate(const orc_problem *P, const uint8_t *policy, int n_rollouts, int horizon,
                 int warmup, uint64_t seed, double *returns, double *kpis, int32_t *traj,
                 int32_t *demand_out);

/* orc_simulate plus per-product KPIs: kpis_prod[6r + 3k + j] = product k's
 * service % (product 1 counts its shortfall met by substitution as served),
 * wastage % of the units received, mean units carried.  NULL skips them. */
int orc_simulate_ex(const orc_problem *P, const uint8_t *policy, int n_rollouts, int horizon,
                    int warmup, uint64_t seed, double *returns, double *kpis, double *kpis_prod,
                    int32_t *traj, int32_t *demand_out);

/* Modified base-stock heuristic (Scenario B "Heuristic policies"): product k
 * orders [S_k - I_k + [X_{1,k} - mu_k]^+]^+ looking at its own stock only, with
 * I_k the units on hand (X_1..X_{m-1} and, when L >= 2, the arrival P_1) and
 * X_{1,k} the units that expire this period; cap != 0 clips the order at Q_k,
 * cap == 0 lets it exceed Q_k (stock is kept as plain vectors, not as a state
 * index).  Same random numbers, reward and KPIs as orc_simulate_ex. */
int orc_mbs_simulate(const orc_problem *P, const int S[2], const int mu[2], int cap, int n_rollouts,
                     int horizon, int warmup, uint64_t seed, double *returns, double *kpis_prod);

/* ---------------------------------------------------------------------------
 * Scenario C (periodic demand, uncertain useful life on arrival; oracle_pc.c).
 * State s = tau (A_max+1)^(m-1) + sum_j X_j (A_max+1)^(j-1): weekday tau
 * (0 = Monday) and X_1..X_{m-1}, the units with j days of life left (X_1
 * expires at the end of today), each 0..A_max.  Actions 0..A_max.
 * ------------------------------------------------------------------------- */
typedef struct {
    int m;                   /* maximum useful life on arrival, 2..8 */
    int Q;                   /* A_max: largest order and capacity for each age */
    int dmax;                /* demand support 0..dmax */
    const double *pmf;       /* 7 x (dmax+1): demand pmf of weekday tau in row tau */
    double c0[9], c1[9];     /* log(p_k(a) / p_1(a)) = c0[k] + c1[k] a, k = 2..m */
    double cost[4];          /* C_f (fixed, per order placed), C_h, C_s, C_w per unit */
    double gamma;            /* 0 < gamma < 1 */
} orc_periodic;

typedef struct {
    long long s_next;
    double reward;
    double demand, issued;
    double wasted;           /* units expiring at the end of the day */
    double held;             /* units left at the end of the day, expiring ones included */
    double accepted;         /* units received into stock */
    double refused;          /* units refused at delivery (age capacity) */
} orc_pc_step;

long long orc_pc_num_states(const orc_periodic *P);
void orc_pc_arrival_params(const orc_periodic *P, int a, double *p);            /* p[1..m] */
double orc_pc_arrival_prob(const orc_periodic *P, int a, const int *y);          /* y[1..m] */
/* next composition y[1..m] of a (start: y_1 = a, others 0); 0 when exhausted */
int orc_pc_next_profile(int m, int a, int *y);
int orc_pc_transition(const orc_periodic *P, long long s, int a, int d, const int *y, orc_pc_step *out);
int orc_pc_qvalues(const orc_periodic *P, const double *V, long long s, double *q);
int orc_pc_backup_states(const orc_periodic *P, const double *V, const long long *states, long long n,
                         double *v_out, int *pol_out, int nthreads);
/* value iteration from V; stop_rule 0 = span, 1 = sup-norm (criterion < eps),
 * 2 = periodic test (Scenario C appendix, tested from i = 7 on).  Returns 0 if
 * converged, 3 at max_iters, 1 on bad input.  dmax/dmin: extremes of V_i - V_{i-1}
 * (rules 0, 1) or of Delta_i (rule 2). */
int orc_pc_vi_solve(const orc_periodic *P, double eps, int stop_rule, int max_iters, double *V, uint8_t *policy,
                    int *iters, double *crit_out, double *dmax_out, double *dmin_out, int nthreads);
/* Rollouts from state 0 (Monday, no stock).  Period t of rollout r: demand from
 * word 0 of Philox4x32-10(ctr (t, r, 0, 0)) by the weekday's thresholds
 * floor(2^32 CDF(d)); unit u of the order takes age class k (1..m) from word
 * u % 4 of Philox4x32-10(ctr (t, r, 1 + u / 4, 0)) by the thresholds
 * floor(2^32 (p_1(a) + .. + p_k(a))).  kpis[3r..] = service %, wastage % of the
 * units accepted, mean units held at the end of the day (expiring included). */
int orc_pc_simulate(const orc_periodic *P, const uint8_t *policy, int n_rollouts, int horizon, int warmup,
                    uint64_t seed, double *returns, double *kpis, int32_t *traj);

#ifdef __cplusplus
}
#endif
#endif
