// vi_api_internal.h -- the handle behind vi_handle (host side only).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "../../include/vi.h"
#include "vi_common.cuh"

struct vi_problem {
    vi_problem_desc desc;              // pmf pointers redirected to the copies below
    std::vector<double> pmf[2];
    vib::KernelParams kp;              // tables / state pointers filled in
    int n_outcomes = 0;                // nominal |Omega|
    int value_bytes = 4;
    int vk = 0;                        // value kind (VK_SINGLE / VK_PAIR / VK_DOUBLE)
    int kahan = 0;                     // compensated sums over outcomes
    bool group_ok = false;             // the factorised kernel can run this instance
    bool two_ok = false;               // the factorised two-product sweep can run this instance
    int kernel_choice = 0;             // VI_KERNEL_AUTO / _GENERIC / _GROUP
    int group_xw = 0;                  // lane width of the factorised kernel (0 = not chosen yet)
    int sweep_xw = 0;                  // kernel of the next launches: 0 generic, else lane width
    int graph_xw = -1;                 // kernel captured in the graph
    int pe_max_iters = 100000;
    // device resources
    float *d_tab_f = nullptr;
    double *d_tab_d = nullptr;
    vib::SolveState *d_state = nullptr;
    vib::SolveState *h_state = nullptr;   // pinned mirror
    void *d_scratch = nullptr;            // second half of the value ping-pong
    float *d_two_e2 = nullptr;            // two-product expectation tables (factorised sweep)
    float *d_two_mix = nullptr;
    uint32_t *d_two_rperm = nullptr;      // rests of product 1 ordered by unit total (pipeline form)
    uint32_t *d_grp_order = nullptr;      // block order of the factorised sweep for lane width order_xw
    int order_xw = 0;
    // periodic problems (Scenario C, vi_pc.cu)
    bool periodic = false;
    double *d_pc_pmf = nullptr;
    unsigned long long *d_pc_prof = nullptr;
    double *d_pc_prob = nullptr;
    int *d_pc_off = nullptr;
    double *d_pc_W = nullptr;
    double *d_pc_ring = nullptr;
    unsigned long long *d_pc_thr_d = nullptr, *d_pc_thr_y = nullptr;
    double *d_pe[2] = {nullptr, nullptr};
    void *d_stage_v = nullptr;            // vi_solve_host staging
    uint8_t *d_stage_p = nullptr;
    cudaStream_t own_stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // solve graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    unsigned long long cond = 0;
    vib::KernelParams args_kp;
    uint32_t args_nS = 0;
    int args_mode_sweep = 0, args_mode_extract = 1;
    int args_lpr = 0;
    void *args_null_v = nullptr;
    uint8_t *args_null_p = nullptr;
};

vi_status vi_fail(vi_status s, const char *fmt, ...);
// Expected one-period reward without the order cost, given y1 units in the
// expiring slot and R in the others (T = y1 + R available), with G[n] = E[(n-D)^+]
// and mu = E[D]:  (c_s + c_r) T - c_s mu - (c_h + c_s + c_r) G[T] + (c_h - c_w) E[W],
// E[W] = G[y1] (FIFO: the expiring units go first) or G[T] - G[R] (LIFO: last).
inline double expected_period_reward(int y1, int R, const double *G, double mu, const double *cost, int issuing) {
    const double c_h = cost[1], c_s = cost[2], c_w = cost[3], c_r = cost[4];
    const int T = y1 + R;
    const double ew = (issuing == VI_LIFO) ? G[T] - G[R] : G[y1];
    return (c_s + c_r) * T - c_s * mu - (c_h + c_s + c_r) * G[T] + (c_h - c_w) * ew;
}
// shared with the allocation-free entry point (vi_noalloc.cu)
void fill_prod_params(vib::ProdParams &P, int m, int L, int Q, int dmax, double c_o);
int heuristic_width(int G, int lifo);
// the solve server's table builder: validates one product of d and fills the
// kernel parameters (no device pointers) and the FP32 table blob
vi_status build_single_product(const vi_problem_desc &d, vib::KernelParams &kp, std::vector<float> &ftab,
                               int &n_outcomes);
