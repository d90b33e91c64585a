/*
 * vi.h -- C ABI of the B300 value-iteration library for perishable-inventory
 * MDPs (Farrington, Li, Wong, Utley, "Going faster to see further:
 * GPU-accelerated value iteration and simulation for perishable inventory
 * control using JAX", 2023).
 *
 * Model.  A single-product instance (m, L, Q, costs, demand pmf, gamma,
 * issuing rule) has states made of the on-hand stock X_1..X_{m-1} split by
 * remaining useful life (X_1 expires at the end of the current period) and
 * the orders in transit P_1..P_{L-1} (P_1 arrives before this period's
 * demand; P_{L-1} is the order placed one period ago).  This is the state of
 * the paper's Scenario A (Appendix A, "Scenario description") observed at the
 * decision epoch, before the arriving units join the stock.  The order a in
 * 0..Q is placed; the arrival u (= P_1 if L >= 2, else a itself) joins as the
 * freshest slot; demand d is issued FIFO (Eq. demoor:fifo) or LIFO
 * (Eq. demoor:lifo); what is left of the oldest slot expires; the rest ages
 * by one period.  Reward (Eq. demoor:reward plus the revenue term of the
 * Scenario B reward):
 *   r = -c_o a - c_h carried - c_s short - c_w wasted + c_r issued.
 * Two products (Scenario B): a shortfall of product 1 is offered product 2,
 * each short unit accepting with probability subst_rate (binomial); product 2
 * serves its own demand first.
 *
 * State index: digit k has weight (Q+1)^k; digits 0..m-2 hold X_1..X_{m-1},
 * digits m-1..m+L-3 hold P_1..P_{L-1}; |S| = (Q+1)^((m-1)+(L-1)).  Two
 * products: s = s_1 + |S_1| s_2 and joint action a = a_1 (Q_2+1) + a_2.
 *
 * Conventions.
 *  - Every function returns vi_status and never aborts the process.
 *  - Pointers documented "device" are CUDA device pointers owned by the
 *    caller; "host" pointers are ordinary host memory owned by the caller.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *  - All scratch (ping-pong value buffer, tables, reduction slots, graphs)
 *    belongs to the handle and is released by vi_problem_destroy.  Released
 *    device blocks (up to 8 GiB), pinned host blocks (up to 256 MiB) and
 *    streams are kept by the library for the next handle of a similar size;
 *    vi_release_cached_memory frees them.
 *  - A handle is not thread-safe; use one handle per host thread.  The solve
 *    server is thread-safe.
 *  - vi_last_error() describes the most recent failure on the calling thread.
 */
#ifndef VI_B300_VI_H
#define VI_B300_VI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vi_problem *vi_handle;
typedef struct vi_server_s *vi_server;

typedef enum {
    VI_OK = 0,
    VI_EINVAL = 1,          /* an argument is out of range (nothing was changed) */
    VI_ENOMEM = 2,          /* device or host allocation failed */
    VI_ENOTCONVERGED = 3,   /* max_iters reached; V and policy hold the last iterate */
    VI_ETIMEOUT = 4,        /* a bounded device-side wait ran out */
    VI_EBUSY = 5,           /* server: request does not fit the memory budget yet */
    VI_ECUDA = 6,           /* a CUDA runtime call failed (see vi_last_error) */
    VI_ECANCELLED = 7       /* work cancelled from the host */
} vi_status;

enum { VI_FIFO = 0, VI_LIFO = 1 };
/* stopping tests: span of V_i - V_{i-1} (Scenario B convergence test) or its
 * sup-norm (Scenario A convergence test); both strict "< tol". */
enum { VI_STOP_SPAN = 0, VI_STOP_SUPNORM = 1, VI_STOP_PERIODIC = 2 };
/* Value arithmetic and storage.
 *  VI_PREC_FP32        FP32 arithmetic; each value is stored as an unevaluated
 *                      pair of floats (hi, lo), V = hi + lo, interleaved as
 *                      float[2|S|].  Sums over outcomes are formed in FP32 from
 *                      differences between values; the absolute value is
 *                      rebuilt with error-free float transformations, so the
 *                      stopping test sees no FP32 rounding noise.
 *  VI_PREC_FP32_KAHAN  as VI_PREC_FP32 with compensated (Kahan) sums over
 *                      outcomes: in the one-thread-per-state kernel
 *                      (VI_KERNEL_GENERIC), which single-product instances run in
 *                      this mode, and in the factorised two-product sweep for lead
 *                      time one on both products (its product-2 expectation and
 *                      substitution-mixture sums and its sum over product-1
 *                      demand).  Two products with longer lead times run the
 *                      generic kernel in this mode (their factorised pipeline
 *                      form is not compensated).
 *  VI_PREC_FP64        FP64 arithmetic and storage, double[|S|].
 *  VI_PREC_FP32_SINGLE one float per state relative to an FP64 offset
 *                      (V = info.offset + v), float[|S|].  Fastest; its stopping
 *                      test is limited by FP32 rounding (about 1e-7 |V|). */
enum { VI_PREC_FP32 = 0, VI_PREC_FP32_KAHAN = 1, VI_PREC_FP64 = 2, VI_PREC_FP32_SINGLE = 3 };

/* vi_solve flags */
enum {
    VI_FLAG_WARM_START = 1,    /* V holds the starting iterate (offset in info->offset) */
    VI_FLAG_NO_GRAPH = 2,      /* host-driven sweep loop instead of the CUDA-graph loop */
    VI_FLAG_POLICY_EVAL = 4    /* after extraction, evaluate the policy in FP64 (see info) */
};

/* Full problem description.  cost[k] = {c_o order, c_h holding, c_s shortage,
 * c_w waste, c_r revenue} per unit for product k (all >= 0).  pmf[k] = host
 * array of dmax[k]+1 probabilities summing to 1 (tail mass already folded into
 * the last entry, as in the paper's truncated demand).  Two products may have
 * any lead times (the paper's Scenario B, where an order arrives before the next
 * day, is L = 2 for both in this convention: the arrival slot P_1). */
typedef struct {
    int n_products;          /* 1 or 2 */
    int m[2], L[2], Q[2];
    double cost[2][5];
    const double *pmf[2];    /* host */
    int dmax[2];
    double subst_rate;       /* product-1 shortfall accepting product 2, in [0,1] */
    double gamma;            /* discount, 0 < gamma <= 1 */
    int issuing;             /* VI_FIFO or VI_LIFO */
    int precision;           /* VI_PREC_* */
    int stop_rule;           /* VI_STOP_* */
} vi_problem_desc;

typedef struct {
    int iters;               /* Bellman sweeps applied (V_iters is returned) */
    int status;              /* VI_OK or VI_ENOTCONVERGED */
    double crit;             /* stopping criterion of the last sweep */
    double dmax, dmin;       /* max / min over s of V_iters(s) - V_{iters-1}(s) (absolute) */
    double offset;           /* FP64 offset b: V_abs(s) = offset + V[s] (VI_PREC_FP32_SINGLE; else 0) */
    double wall_ms;          /* device time of the solve (CUDA events), sweeps + extraction */
    double updates_per_s;    /* nominal |S||A||Omega| x iters / wall time */
    int pe_iters;            /* FP64 policy-evaluation sweeps (VI_FLAG_POLICY_EVAL; a multiple of 8) */
    double pe_delta;         /* last sup-norm change of the policy evaluation */
    double pe_gap;           /* max_s |V_pe(s) - V_abs(s)| after evaluation */
    double pe_span;          /* max_s - min_s of V_pe(s) - V_abs(s): the gap up to a constant,
                                the relevant one after a span-test stop */
} vi_solve_info;

/* Create a single-product problem (VI_PREC_FP32, span stopping test).
 * Defines: state space and transition of Scenario A (Appendix A, state
 * definition, Eq. demoor:fifo / demoor:lifo, Eq. demoor:reward).
 * cost: host double[5]; pmf: host double[dmax+1].  Copies everything it needs
 * to the current CUDA device.  Errors: VI_EINVAL for m < 1, L < 1, Q < 0,
 * Q+1 > 256 (policy is uint8), |S| >= 2^32, dmax < 0 or > 4095, pmf entries
 * < 0 or not summing to 1 within 1e-12, gamma outside (0, 1], a negative cost
 * or issuing not FIFO/LIFO; VI_ENOMEM / VI_ECUDA on allocation failure. */
vi_status vi_problem_create(int m, int L, int Q, const double cost[5], const double *pmf,
                            int dmax, double gamma, int issuing, vi_handle *out);

/* Create a problem from a full description (one or two products, precision,
 * stopping rule).  Same errors as vi_problem_create; two products also need
 * |A| = (Q_1+1)(Q_2+1) <= 256, dmax <= 255 and subst_rate in [0,1]. */
vi_status vi_problem_create_desc(const vi_problem_desc *desc, vi_handle *out);

/* Scenario C of the paper (Scenario C appendix): weekday-periodic demand and
 * uncertain useful life on arrival.  State s = tau (Q+1)^(m-1) + sum_j X_j
 * (Q+1)^(j-1): the weekday tau (0 = Monday) and X_1..X_{m-1}, the units with j
 * days of life left (X_1 expires at the end of today), each 0..Q; actions
 * 0..Q.  An order a arrives at once as y_1..y_m units with k days left,
 * multinomial over the a units with log(p_k(a) / p_1(a)) = c0[k] + c1[k] a
 * (Eq. mirjalili:ageonarrival); units beyond Q of an age are refused at
 * delivery; the day's demand (pmf row tau, Eq. mirjalili:demand) is issued
 * oldest first (Eq. mirjalili:state_transition); reward -C_f 1{a > 0} - C_h
 * (units left, expiring ones included) - C_s (unmet demand) - C_w (expiring
 * units left).  Solved in FP64 (V: device double[|S|] in vi_solve), with
 * stop_rule VI_STOP_PERIODIC the periodic test of the appendix (for i >= 7,
 * Delta_i(s) = sum_{j=0}^{6} gamma^-(i-j-1) (V_{i-j}(s) - V_{i-j-1}(s)); stop at
 * max Delta - min Delta <= 2 tol min(|max Delta|, |min Delta|); vi_solve_info
 * dmax/dmin then report max/min Delta and crit their relative spread).
 * vi_simulate draws the day's demand from word 0 of Philox4x32-10(ctr (t, r, 0,
 * 0)) by the weekday's floor(2^32 CDF) thresholds and unit u of the order's age
 * class from word u % 4 of Philox4x32-10(ctr (t, r, 1 + u / 4, 0)) by the
 * thresholds floor(2^32 (p_1(a) + .. + p_k(a))); kpis = service %, wastage % of
 * the units accepted, mean units left at the end of the day (expiring
 * included).  vi_simulate_ex needs kpis_prod = NULL; vi_policy_eval,
 * VI_FLAG_POLICY_EVAL, vi_next_states and the base-stock searches return
 * VI_EINVAL for these problems. */
typedef struct {
    int m;                   /* maximum useful life on arrival, 2..8 */
    int Q;                   /* A_max: largest order and capacity of each age, 0..63 */
    int dmax;                /* demand support 0..dmax */
    const double *pmf;       /* host, 7 x (dmax+1), row tau = weekday tau's demand pmf */
    double c0[9], c1[9];     /* logits of the life on arrival, entries 2..m used */
    double cost[4];          /* C_f per order placed, C_h, C_s, C_w per unit (>= 0) */
    double gamma;            /* 0 < gamma < 1 */
    int stop_rule;           /* VI_STOP_PERIODIC, VI_STOP_SPAN or VI_STOP_SUPNORM */
} vi_periodic_desc;

/* Create a Scenario C problem.  Copies everything it needs to the current
 * device.  Errors: VI_EINVAL for m outside 2..8, Q outside 0..63, a pmf row not
 * summing to 1 within 1e-12, gamma outside (0, 1), a negative cost, a bad stop
 * rule or 7 (Q+1)^m >= 2^31; VI_ENOMEM / VI_ECUDA. */
vi_status vi_problem_create_periodic(const vi_periodic_desc *desc, vi_handle *out);

/* Release every device and host resource of the handle.  NULL is accepted.
 * Synchronises the current device first (as cudaFree does): the handle's
 * blocks then go to the library's cache of blocks (see Conventions). */
vi_status vi_problem_destroy(vi_handle h);

/* Free every cached device block, pinned host block and idle stream that
 * destroyed handles left to the library (no counterpart in the paper; memory
 * management).  *bytes_released (may be NULL) receives the bytes freed.  Call
 * it when no handle is being created or destroyed on another thread. */
vi_status vi_release_cached_memory(size_t *bytes_released);

/* Bytes currently held in that cache (device plus pinned host).
 * Errors: VI_EINVAL for a NULL pointer. */
vi_status vi_cached_memory(size_t *bytes);

/* Sizes: |S|, |A|, nominal |Omega| and bytes per stored value (4 for
 * VI_PREC_FP32_SINGLE, else 8). */
vi_status vi_problem_sizes(vi_handle h, uint64_t *n_states, int *n_actions,
                           int *n_outcomes, int *value_bytes);

/* Per-handle options (no counterpart in the paper; tuning and test hooks).
 * VI_OPT_KERNEL: which sweep kernel runs -- VI_KERNEL_AUTO (factorised kernel
 * whenever the instance allows it; for LIFO with L = 1 the VI_KERNEL_LIFO_L1
 * sweep and for FIFO the VI_KERNEL_FIFO_COL sweep is one of the autotuned
 * candidates; two products in VI_PREC_FP32 run the factorised
 * two-product sweep -- with lead times >= 2 on both products its pipeline form
 * (m >= 2, Q+1 <= 32) -- which vi_problem_kernel reports as VI_KERNEL_GROUP with
 * width 0),
 * VI_KERNEL_GENERIC (one thread per state),
 * VI_KERNEL_GROUP (factorised; VI_EINVAL if the instance does not allow it:
 * it needs one product, VI_PREC_FP32 or VI_PREC_FP32_SINGLE, 2 <= Q+1 <= 64 and
 * at least one state digit) or VI_KERNEL_TENSOR (factorised, with the FIFO
 * expectation of a tile of rests and orders computed as one product on the
 * tensor cores; VI_EINVAL unless one product, FIFO, VI_PREC_FP32, L >= 2,
 * 2 <= Q+1 <= 32 and Dmax <= 127; only run when asked for) or
 * VI_KERNEL_LIFO_L1 (factorised LIFO sweep for lead time one: every order's
 * next states lie on two sequences of the rest -- the order partly used, the
 * order used up and the rest issued freshest first -- gathered once per rest,
 * so each order's expectation is a short convolution of them with the pmf; the
 * used-up part carried from rest to rest along the rests that differ only in
 * the freshest rest slot (the first one issued after the order); persistent
 * blocks; VI_EINVAL unless one product, LIFO, VI_PREC_FP32, L = 1,
 * m >= 2, 2 <= Q+1 <= 16 and Dmax <= 31) or
 * VI_KERNEL_FIFO_COL (FIFO sweep by columns of rests: the Q+1 rests that
 * differ only in the oldest rest slot Z_1 share one expectation over the
 * demand, from which each rest's follows by one multiply-add per
 * (expiring-slot value, order), since one unit more in Z_1 is the first to be
 * issued after the expiring slot; one of the autotuned candidates; VI_EINVAL
 * unless one product, FIFO, VI_PREC_FP32, m >= 2 (m >= 3 with L = 1),
 * 2 <= Q+1 <= 32 and Dmax <= 62).
 * VI_OPT_PE_MAX_ITERS: sweep cap of the FP64 policy evaluation in vi_solve.
 * VI_OPT_GROUP_WIDTH: run the factorised kernel with this many expiring-slot
 * values per lane (1..12, 16, 21 or 24; Q+1 is split over ceil((Q+1)/width)
 * lanes).  Without it the width is autotuned on the first solve (one timed
 * sweep per candidate width, cached per instance shape; the environment
 * variable VI_AUTOTUNE=0 selects a fixed rule instead).
 * VI_OPT_TEST_STALL (test hook): 1 makes the tensor-core kernel withhold its
 * MMAs, so that its bounded wait for them runs out after a short limit; the
 * sweep then reports VI_ECUDA ("bounded wait ... gave up") and the CUDA
 * context stays usable.  0 restores normal operation. */
enum { VI_OPT_KERNEL = 1, VI_OPT_PE_MAX_ITERS = 2, VI_OPT_GROUP_WIDTH = 3, VI_OPT_TEST_STALL = 4 };
enum {
    VI_KERNEL_AUTO = 0,
    VI_KERNEL_GENERIC = 1,
    VI_KERNEL_GROUP = 2,
    VI_KERNEL_TENSOR = 3,
    VI_KERNEL_LIFO_L1 = 4,
    VI_KERNEL_FIFO_COL = 5
};
vi_status vi_problem_set_option(vi_handle h, int option, int value);

/* Which sweep kernel the handle runs (no counterpart in the paper): *kernel =
 * VI_KERNEL_GENERIC, VI_KERNEL_GROUP, VI_KERNEL_TENSOR, VI_KERNEL_LIFO_L1 or
 * VI_KERNEL_FIFO_COL,
 * *width = the lane width of VI_KERNEL_GROUP (0 otherwise).  Resolves the choice (and runs the
 * autotuner, on the handle's default stream) if no solve has done so yet.
 * Either pointer may be NULL.  Errors: VI_EINVAL (null handle), VI_ECUDA. */
vi_status vi_problem_kernel(vi_handle h, int *kernel, int *width);

/* Synchronous value iteration (Eq. valueiterationdetupdate, Algorithm 1) from
 * V_0 = 0 (or the warm start), stopping at the first i with the stopping
 * criterion < tol, or at max_iters; then one extraction sweep writes the
 * first argmax policy from V_i (Eq. valueiterationdetpolicy, Algorithm 1).
 * V: device buffer in the precision's layout (float[2|S|] pairs for
 * VI_PREC_FP32 / _KAHAN, double[|S|] for VI_PREC_FP64, float[|S|] plus
 * info->offset for VI_PREC_FP32_SINGLE), in/out.  policy: device uint8[|S|] or NULL.
 * info: host, out (and in: offset when VI_FLAG_WARM_START).  Blocks until the
 * solve is done.  Returns VI_OK, VI_ENOTCONVERGED (V/policy hold the last
 * iterate), VI_EINVAL (max_iters < 0, tol < 0, V NULL) or VI_ECUDA. */
vi_status vi_solve(vi_handle h, double tol, int max_iters, void *V, uint8_t *policy,
                   void *stream, int flags, vi_solve_info *info);

/* vi_solve on host buffers: copies the warm start (if any) host->device,
 * solves, and returns V and the policy in the host buffers.  V_host: host buffer
 * in the precision's layout (see vi_solve) holding |S| values; policy_host: host
 * uint8[|S|] or NULL.  When every given host buffer is page-locked
 * (cudaMallocHost, cudaHostAlloc, cudaHostRegister) and VI_FLAG_POLICY_EVAL is
 * not set, the extraction sweep writes V and the policy into them directly, so
 * the transfer overlaps the sweep; otherwise they are copied from device
 * staging buffers after it.  Staging buffers are owned by the handle
 * (allocated on first use). */
vi_status vi_solve_host(vi_handle h, double tol, int max_iters, void *V_host,
                        uint8_t *policy_host, int flags, vi_solve_info *info);

/* One Bellman sweep without renormalisation: V_out(s) = max_a [rbar(s,a) +
 * gamma sum_omega P(omega) V_in(s'_omega)] and policy(s) = first argmax
 * (Eq. valueiterationdetupdate).  VI_PREC_FP32_SINGLE: if V_in holds V_abs - b
 * then V_out holds V_abs' - gamma b.  V_in/V_out: device buffers in the
 * precision's layout (must differ);
 * policy: device uint8[|S|] or NULL; dstats: host double[2] or NULL, receives
 * max and min of V_out - V_in.  Synchronises the stream when dstats != NULL. */
vi_status vi_backup(vi_handle h, const void *V_in, void *V_out, uint8_t *policy,
                    void *stream, double *dstats);

/* Evaluate a fixed policy in FP64 (the paper's double-precision arithmetic,
 * Methods "Value iteration"): V <- r_pi + gamma P_pi V until the sup-norm
 * change is < tol or max_iters sweeps.  The change is read back after every
 * 8th sweep (and after sweep max_iters), so iters is the first multiple of 8
 * at or past the sweep whose change fell below tol, and delta is the change of
 * that sweep.  V: device double[|S|], in (start) / out.  policy: device
 * uint8[|S|].  iters / delta: host out (may be NULL).  Returns VI_OK or
 * VI_ENOTCONVERGED. */
vi_status vi_policy_eval(vi_handle h, const uint8_t *policy, double *V, double tol,
                         int max_iters, void *stream, int *iters, double *delta);

/* Next-state indices T(s, a, omega) of the listed states, computed with the
 * same incremental index arithmetic as the sweep kernels (Eq. demoor:fifo /
 * demoor:lifo).  states: device uint32[n].  out: device uint32, single product
 * n x |A| x (dmax+1) laid out [i][a][d]; two products n x |A| x (dmax1+1) x
 * (dmax1+dmax2+1) laid out [i][a][d1][z] where z = units of demand facing
 * product 2 (own demand plus accepted substitutes). */
vi_status vi_next_states(vi_handle h, const uint32_t *states, int n, uint32_t *out, void *stream);

/* Policy rollouts (the paper's simulators, Methods "Simulation of the Markov
 * decision processes"): n_rollouts independent runs from the all-zero state;
 * period t of rollout r draws Philox4x32-10 with counter (t, r, 0, 0) and key
 * (seed low 32 bits, seed high 32 bits); word 0 is turned into product-1
 * demand by the integer inverse CDF (smallest d with word < floor(2^32 CDF(d)),
 * CDF summed in ascending order in FP64), word 1 into product-2 demand, and
 * the popcount of the low `shortfall` bits of the 64-bit word (word 3, word 2)
 * gives the accepted substitutions (two products need subst_rate = 1/2; a
 * shortfall above 64 uses all 64 bits).  The first `warmup`
 * periods are simulated but not scored.  policy: device uint8[|S|], entries
 * below |A|;
 * returns: device double[n] = sum_t gamma^t r_t (FP64, in period order);
 * kpis: device double[3n] or NULL = {service %, wastage %, mean units carried};
 * traj: device int32[n x horizon] or NULL = state before each scored decision. */
vi_status vi_simulate(vi_handle h, const uint8_t *policy, int n_rollouts, int horizon,
                      int warmup, uint64_t seed, double *returns, double *kpis,
                      int32_t *traj, void *stream);

/* vi_simulate plus per-product KPIs (Scenario B appendix, KPI tables):
 * kpis_prod: device double[6n] or NULL; entry 6r + 3k + j is, for product k
 * of rollout r, j = 0 the service level % (product 1's shortfall met by
 * substitution counts as served), j = 1 wastage % of the units received, j = 2
 * mean units carried to the next period.  Product index 1 is {100, 0, 0} for
 * one product.  Other arguments and errors as vi_simulate. */
vi_status vi_simulate_ex(vi_handle h, const uint8_t *policy, int n_rollouts, int horizon, int warmup,
                         uint64_t seed, double *returns, double *kpis, double *kpis_prod, int32_t *traj,
                         void *stream);

/* Modified base-stock search by simulation (Scenario B "Heuristic policies",
 * after Haijema et al.): product k orders [S_k - I_k + [X_{1,k} - mu_k]^+]^+,
 * I_k = its units on hand (X_1..X_{m-1} and the arrival P_1 when L >= 2),
 * X_{1,k} = its units expiring this period; cap != 0 clips each order at Q_k,
 * cap == 0 lets it exceed Q_k (the simulation keeps plain slot counts).  Every
 * pair (S_1, S_2) in [S_lo, S_hi] (S_lo[1], S_hi[1], mu[1] ignored for one
 * product) runs n_rollouts rollouts from empty stock with `warmup` unscored
 * periods and `horizon` scored ones, on the random numbers of vi_simulate.
 * returns: device double[n_pairs * n_rollouts], row pair = (S_1 - S_lo[0]) *
 * n_2 + (S_2 - S_lo[1]); kpis_prod: device double[6 n_pairs n_rollouts] or
 * NULL (layout of vi_simulate_ex); mean_returns: host double[n_pairs] or NULL;
 * best_S: host int[2] or NULL (the first pair with the largest mean, FP64
 * sums in rollout order; the stream is synchronised when either is given).
 * Errors: VI_EINVAL (bad ranges, m > 8 or L > 4, dmax above the rollout limit,
 * subst_rate other than 1/2 for two products), VI_ECUDA. */
vi_status vi_mbs_search(vi_handle h, const int S_lo[2], const int S_hi[2], const int mu[2], int cap,
                        int n_rollouts, int horizon, int warmup, uint64_t seed, double *returns,
                        double *kpis_prod, double *mean_returns, int best_S[2], void *stream);

/* Base-stock policy search by simulation (Methods, Scenario A heuristic policy:
 * A = [S - I]^+ with I the total stock on hand and in transit; the paper scores
 * every S in 0..A_max by its mean simulated return).  Single product.  For each
 * S in s_lo..s_hi, n_rollouts rollouts from the all-zero state with `warmup`
 * unscored periods then `horizon` scored ones, exactly as vi_simulate does with
 * the policy A(s) = min([S - I(s)]^+, Q); every S uses the same random numbers
 * (Philox counters (t, r)).
 * returns: device double[(s_hi - s_lo + 1) * n_rollouts], row S - s_lo, column r
 * (the caller's buffer).  mean_returns: host double[s_hi - s_lo + 1] or NULL;
 * best_S: host int or NULL (the first S with the largest mean); when either is
 * given the stream is synchronised and the means are summed in FP64 in rollout
 * order.  Errors: VI_EINVAL (two products, bad sizes, dmax above the rollout
 * limit), VI_ECUDA. */
vi_status vi_basestock_search(vi_handle h, int s_lo, int s_hi, int n_rollouts, int horizon, int warmup,
                              uint64_t seed, double *returns, double *mean_returns, int *best_S, void *stream);

/* Continuous-batching solve server (no counterpart in the paper; it serves the
 * paper's value iteration to many callers).  Requests -- single-product
 * instances with 2 <= Q+1 <= 24 and at least one state digit, solved in
 * VI_PREC_FP32 with the span stopping test -- wait in arrival order and are
 * admitted while a slot is free and their device memory (about 17 bytes per
 * state) fits mem_budget_bytes.  A host worker thread with its own stream keeps
 * one persistent kernel launch running over all admitted instances: its blocks
 * claim blocks of the instances' current sweeps (largest instances first), and
 * each instance's next sweep -- or its extraction sweep once its stopping test
 * has passed -- starts as soon as its previous one has finished, so instances of
 * different sizes advance together, each at its own pace.  FIFO instances that
 * VI_KERNEL_FIFO_COL accepts, with Dmax <= 46, run its body, the others
 * that of VI_KERNEL_GROUP, so a result equals, bit for bit, the instance solved
 * alone with that kernel.  A finished instance
 * is retired between launches, freeing memory for queued requests; its values
 * and policy are copied to host memory by retirement threads.  Value buffers
 * come from a memory pool of the server's own that keeps freed memory reserved
 * up to the budget (min(budget, 1 GiB) is reserved at creation).  `stream` is
 * unused (the worker owns a stream); max_slots in 1..1024. */
vi_status vi_server_create(size_t mem_budget_bytes, int max_slots, void *stream, vi_server *out);
/* Queue a request; returns at once with its id.  The description is copied.
 * VI_EINVAL for a bad description, VI_EBUSY if it can never fit the budget. */
vi_status vi_server_submit(vi_server srv, const vi_problem_desc *desc, double tol, int max_iters,
                           uint64_t *request_id);
/* vi_server_submit that delivers the result into the caller's host buffers:
 * V_host (double[|S|], absolute values) and policy_host (uint8[|S|]) are
 * written by the server's retirement threads before the request reports done,
 * so the caller copies nothing; they must stay valid until then.  Either may be
 * NULL (that part then waits in the server for vi_server_poll).  Errors as
 * vi_server_submit. */
vi_status vi_server_submit_to(vi_server srv, const vi_problem_desc *desc, double tol, int max_iters,
                              double *V_host, uint8_t *policy_host, uint64_t *request_id);
/* Poll a request.  done = 1 once finished; then V_host (host double[|S|],
 * absolute values, or NULL) and policy_host (host uint8[|S|] or NULL) receive
 * the result and info the solve record (wall_ms = submit-to-result latency,
 * updates_per_s over the time the request held a slot).  Returns the request's
 * status (VI_OK, VI_ENOTCONVERGED, VI_ECANCELLED, ...) once done, VI_OK while
 * pending, VI_EINVAL for an unknown id.  A finished request is forgotten after
 * it has been polled as done. */
vi_status vi_server_poll(vi_server srv, uint64_t request_id, int *done, double *V_host,
                         uint8_t *policy_host, vi_solve_info *info);
/* Wait up to timeout_ms (0: do not wait) for requests to finish.  Writes into
 * ids (host uint64[max_ids]) the ids of up to max_ids requests that finished
 * and were not yet reported by this call, in the order they finished, and
 * their count into *n_out (0 after a time-out).  A reported request is then
 * read with vi_server_poll.  VI_EINVAL for bad arguments. */
vi_status vi_server_wait(vi_server srv, int timeout_ms, uint64_t *ids, int max_ids, int *n_out);
/* Stop the worker and release everything.  Pending requests are cancelled. */
vi_status vi_server_destroy(vi_server srv);

/* One Bellman sweep that allocates no memory -- the paper has no counterpart;
 * this entry point exists for callers that cannot allocate when they need a
 * sweep: code running inside an allocator or a memory pool that must not be
 * re-entered, components whose device memory is budgeted by someone else, or
 * callers that reserved everything up front.  It computes what vi_backup
 * computes for a VI_PREC_FP32 single-product problem (V_out(s) = max_a Q(s, a)
 * from V_in, first argmax in policy, max / min of V_out - V_in in dstats)
 * without creating a handle.
 * Arguments: the instance as for vi_problem_create; V_in / V_out: device
 * float-pair buffers (float[2|S|], the VI_PREC_FP32 layout), distinct;
 * policy: device uint8[|S|] or NULL; dstats: host double[2] or NULL (when
 * given, the stream is synchronised); stream: cudaStream_t or NULL.
 * Scratch: the expectation tables and the reduction slots live in a fixed
 * array in device memory that belongs to the library, holding at most
 * VI_NOALLOC_MAX_TABLE_FLOATS table entries (3 (dmax + 1 + mQ + 2(Q+1) + 34)
 * + 2 (Q+1)((m-1)Q + 1) are needed); larger instances get VI_EINVAL.  Every
 * GPU that loads the library holds this array (about 65 KiB) until the
 * process exits.  All calls share it and it keeps the last call's contents
 * (the call resets what must start at zero), so calls whose work overlaps on
 * the GPU -- on different streams, or from several host threads without
 * ordering -- race.  The first call on a device looks up the array's device
 * address (a one-time set-up for that device); make that first call before
 * any stream capture.  A call on a stream that is being captured is refused
 * with VI_EINVAL: the tables go up from a host staging buffer that the next
 * call overwrites.  The address is kept for the life of the process, so
 * the device's primary context must not be reset (cudaDeviceReset) between
 * calls.  No cudaMalloc, cudaFree or other allocator is called.
 * Errors: VI_EINVAL (bad instance or buffers, tables too large, stream being
 * captured), VI_ECUDA. */
#define VI_NOALLOC_MAX_TABLE_FLOATS 16384
vi_status vi_backup_noalloc(int m, int L, int Q, const double cost[5], const double *pmf, int dmax,
                            double gamma, int issuing, const void *V_in, void *V_out, uint8_t *policy,
                            double *dstats, void *stream);

/* Measurement helper (the paper has no counterpart): read bandwidth of the L2
 * cache, the denominator of the gather roofline.  Streams the caller's device
 * buffer `reps` times with 16-byte loads that bypass L1, after one untimed pass
 * that brings it into L2, and returns the timed pass's duration in *ms (CUDA
 * events on `stream`; the call synchronises the stream).  Choose `bytes` well
 * below the L2 size (e.g. 32 MiB of 126 MB) so that the passes hit L2; the read
 * rate is bytes * reps / ms.  The buffer is only read.
 * Errors: VI_EINVAL (NULL, unaligned or too small buffer, reps < 1), VI_ECUDA. */
vi_status vi_probe_l2_read(const void *buf, size_t bytes, int reps, void *stream, float *ms);

const char *vi_status_string(vi_status s);
const char *vi_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* VI_B300_VI_H */
