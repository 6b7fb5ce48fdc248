// Launch arguments and launchers of the FTKomega kernels (host <-> device).
#pragma once
#include "ftk_common.cuh"

#include <string>

namespace ftk {

enum { EPI_PLAIN = 0, EPI_TPQ = 1, EPI_COCG = 2, EPI_COCG_MIXED = 3, EPI_TAYLOR = 4 };

struct EpiArgs {
    const double *scale;     // TPQ: device s_k
    double ell, inv_n;       // TPQ: l, 1/N
    double *partials;        // [grid][nd] scratch
    unsigned int *counter;   // last-block ticket (reset by the last block)
    double *result;          // reduced dots [nd]
    TpqState *tpq;           // TPQ state (updated by the last block)
    double *stat_u, *stat_logq, *stat_h2;   // TPQ statistics arrays [k]
    const int *all_done;     // COCG: skip when every RHS finished (or NULL)
    const void *lo;          // COCG, mixed mode: float2 low parts of the input (mu from hi + lo)
    // Taylor term of the cTPQ series (Appendix A, FP64, one vector):
    // out = tcoef (l v - H v / N), taylor_acc += out; dots <v|H v>, |acc|^2
    double2 *taylor_acc;
    double tcoef;
    long long df_lo;         // double-float mode: float2 offset of the lo arrays of in and out
    // Double-float mode, first pass of H r_{k+1}: the COCG residual update
    // fused in (fu_seed != NULL). Per launch (one column): the pass's input
    // r_{k+1} is computed tile by tile from r_k (fu_rcur), r_{k-1} (in place
    // of which r_{k+1} is written: fu_rnew, the pass's `in`), w_k = H r_k (the
    // pass's `out`, read before it is overwritten) and lambda split
    // (fu_lam); rho, g, |r|^2 of r_{k+1} go to fu_result[0..5). Every pass
    // of a column whose fu_seed is done returns at once.
    // Relaxed double-float solve: the launch runs only while *lowp equals
    // lowp_run (lowp NULL: always)
    const int *lowp;
    int lowp_run;
    const CocgSeed *fu_seed;
    float2 *fu_rcur;
    float2 *fu_rnew;
    const float4 *fu_lam;
    double *fu_result;
};

struct UpdArgs {
    int mode;                // 0: r = lambda, 1: 3-term update
    uint64_t dim;
    const void *lambda[FTK_MAX_RHS];
    // projection vector of g = proj^dag r (the A of <A|(z - H)^-1|B>, Sec. II.B);
    // NULL: the right-hand side itself. Mixed / double-float modes: mode 0
    // writes the split of proj (not of lambda) to lam_split.
    const void *proj[FTK_MAX_RHS];
    const CocgSeed *seed;
    double *partials;
    unsigned int *counter;
    double *result;          // [B][FTK_UPD_DOTS]
    const int *all_done;
    long long lo_stride;     // mixed / double-float: float2 offset of the lo parts from the hi parts
    long long w_lo;          // double-float mode: float2 offset of w's lo part (0: w is float)
    float4 *lam_split;       // mixed / double-float: lambda as (hi.re, hi.im, lo.re, lo.im), [B][dim];
                             // written by mode 0, read by mode 1
    const int *lowp;         // relaxed solve: run only while *lowp == lowp_run (NULL: always)
    int lowp_run;
};

struct SeedArgs {
    int n_rhs;
    int max_iter;
    double tol;
    CocgSeed *seed;
    const double *upd;       // [B][FTK_UPD_DOTS]
    const double *hv;        // [B][FTK_HV_DOTS]
    double *inv_pi_max;      // [2][FTK_MAX_RHS] parity double buffer
    int *all_done;
    double relax;            // relaxed solve: theta (0: off)
    int *lowp;               // set (sticky) once every running RHS has resid < theta
    // seed switching (seed_switch = 1): the shift offsets and the shift state
    // of the block, read when the seed has converged before the other shifts
    int seed_switch;
    int n_omega;
    const struct dcx *shift;            // [n_omega] z_s - E_j (complex offsets)
    const struct dcx *pi_prev, *pi_cur; // [B][n_omega]
    const int *frozen;                  // [B][n_omega]
};

// Shift s of right-hand side j is z_js = E_j + shift[s] (complex; the
// spectrum solves use shift[s] = omega_s + i eta, the contour filter
// E_m + eps e^{i theta} - E_j).
struct ShiftArgs {
    int n_omega;
    const struct dcx *shift; // [n_omega]
    const CocgSeed *seed;
    struct dcx *pi_prev, *pi_cur, *ptil, *G;   // [B][n_omega]
    double *inv_pi_max;      // [2][FTK_MAX_RHS]
    int *frozen;             // [B][n_omega] converged shifts
    double tol;
    // history of the shift recurrences (right-hand side 0 only; NULL: off):
    // per iteration k and shift s, (alpha^s_k, beta^s_{k-1}, 1/pi^s_k) with
    // alpha^s_k = 0 when the shift no longer contributes; hist_cap iterations
    struct dcx *hist;
    int hist_cap;
};

// Seed switch: scale r_k, w_k by s1 and r_{k-1} by s0 for every right-hand
// side whose seed switched in this iteration (CocgSeed::sw), and pi_k,
// pi_{k-1} of all its shifts likewise. kind as launch_cocg_update.
struct SwitchArgs {
    int kind;
    uint64_t dim;
    void *rcur, *rprev, *w;
    long long lo_stride;     // mixed / double-float: float2 offset of the lo parts
    long long w_lo;          // double-float: lo part of w (0: w is float)
    CocgSeed *seed;
    struct dcx *pi_prev, *pi_cur;
    int n_omega;
    const int *all_done;
};

// Contour filter, second pass: phi_m += C[k][m] r_k for every shell centre
// m < L (one right-hand side, FP64 vectors), k = the current iteration.
struct FilterAccArgs {
    uint64_t dim;
    int L;
    int n_coef;              // iterations in coef (a later iteration adds nothing)
    const double2 *r;        // r_k
    double2 *phi;            // [L][dim]
    const struct dcx *coef;  // [iterations][L]
    const CocgSeed *seed;    // iteration index and status of the solve
};

// Contour filter, coefficients: from the recorded history, per shift s the
// backward sum T^s_k = alpha^s_k + beta^s_k T^s_{k+1} (beta^s_k = the
// beta^s of iteration k + 1), C^s_k = T^s_k / pi^s_k, and per centre m
// C[k][m] = sum_{j < M} w_j C^{(m, j)}_k with shift index s = m M + j.
// Reweighting of filter shells (Eqs. FRW1, FRW2), one CTA per temperature:
//   S(omega, T) = sum_m e^{(b - b')E_m} (-Im G_m(omega) / pi) / sum_l e^{(b - b')E_l} n_l
//   P_b'(E_m)   = e^{(b - b')E_m} n_m / (2 eps sum_l e^{(b - b')E_l} n_l)
// with b' = 1/T, n_m = <phi^m|phi^m>, log-sum-exp in double.
struct FrwArgs {
    int n_shell, n_omega;
    double beta, eps;
    const double *E, *norm2;   // [n_shell]
    const double *G;           // [n_shell][n_omega][2]
    const double *T;           // [n_T]
    double *S;                 // [n_T][n_omega]
    double *P;                 // [n_T][n_shell]
};
cudaError_t launch_frw_spectrum(const FrwArgs &fa, int n_T, cudaStream_t st);

struct FilterCoefArgs {
    int n_iter;              // iterations recorded
    int L, M;
    const struct dcx *hist;  // [n_iter][L M][3]
    const struct dcx *w;     // [M] quadrature weights rho e^{i theta_j} / M
    struct dcx *tsum;        // [L M] scratch: T^s of the running iteration
    struct dcx *coef;        // [n_iter][L]
};

struct OpArgs {
    int n_sites;
    int gamma;
    uint64_t dim;
    double f_re[FTK_MAX_SITES], f_im[FTK_MAX_SITES];   // N^{-1/2} exp(i q.R_l)
    const double *scale;     // device scale of the source vector
    double *partials;
    unsigned int *counter;
    double *result;
    const double *energy_src; // device u_k of the source shell (or NULL)
    double n_sites_d;
    double energy_val;
    double *slot_energy;     // device shift origin of the slot
    double *slot_norm2;      // device ||lambda||^2
};

struct InitArgs {
    uint64_t dim;
    uint64_t seed;
    uint32_t sample;
    double *partials;
    unsigned int *counter;
    double *result;
    TpqState *tpq;
};

struct SpecArgs {
    int n_sites_i;
    double n_sites;
    double ell;
    int n_steps;             // K: statistics for k = 0..K-1
    int save_every;
    int n_shell;
    int n_omega;
    const double *u, *logq;  // [K]
    const double *G;         // [n_shell][n_omega][2]
    const double *T;         // [n_T]
    double *S;               // [n_T][n_omega]
    int *trunc;              // [n_T]
};

cudaError_t init_kernel_attributes();
void set_thread_error(const char *msg);   // message for ftk_last_error(NULL)
// What the momentum-sector code reads from a context.
struct CtxHam {
    int n, nb;
    const int *bonds;        // [nb][3]: i, j, gamma
    double K, J, ell_min;
    const double *pos;       // [n][2]
    cudaStream_t stream;
    int n_sm;
    int64_t *launches;       // the context's launch counter
    std::string *err;        // the context's last error message
};
}  // namespace ftk
struct ftk_ctx;
namespace ftk {
bool ctx_hamiltonian(ftk_ctx *c, CtxHam *h);
// H.V pass (ftk_hv.cu). A planned pass is laid out once for the kernel's
// thread layout and a column chunk width cols <= hv_max_b(prec)
// (hv_layout_pass); a launch of B right-hand sides then runs B / cols column
// chunks. grid_cap bounds the persistent grid (the size of ea.partials).
cudaError_t launch_hv_pass(int prec, int B, int epi, const void *in, void *out, const PassDesc &pd,
                           const EpiArgs &ea, int grid_cap, cudaStream_t st);
bool hv_layout_pass(PassDesc &pd, int prec, int B);
int hv_max_b(int prec);
int hv_le(int prec, int B, int tile_bits, int chunk_bits);
int hv_max_tile_bits(int prec, int B);
int hv_threads(const PassDesc &pd);
size_t hv_smem_bytes(int prec, int B, const PassDesc &pd);
// kind: 0 FP64 vectors, 1 FP32 vectors, 2 mixed (split float hi + lo
// residuals, float w, double lambda)
cudaError_t launch_cocg_update(int kind, int B, void *rcur, const void *w, void *rprev_new,
                               const UpdArgs &ua, int grid, cudaStream_t st);
cudaError_t launch_cocg_seed(const SeedArgs &sa, cudaStream_t st);
cudaError_t launch_cocg_shift(const ShiftArgs &sh, int n_rhs, cudaStream_t st);
cudaError_t launch_cocg_switch(const SwitchArgs &sw, int B, int grid, cudaStream_t st);
cudaError_t launch_filter_acc(const FilterAccArgs &fa, int grid, cudaStream_t st);
cudaError_t launch_filter_coef(const FilterCoefArgs &fc, cudaStream_t st);
cudaError_t launch_apply_op(int prec, const void *psi, void *lam, const OpArgs &oa, int grid,
                            cudaStream_t st);
cudaError_t launch_init_state(int prec, void *v, const InitArgs &ia, int grid, cudaStream_t st);
cudaError_t launch_norm(int prec, const void *v, const InitArgs &ia, int grid, cudaStream_t st);
cudaError_t launch_convert_in(int prec, const void *src, void *dst, uint64_t n, int grid, cudaStream_t st);
cudaError_t launch_convert_out(int prec, const void *src, void *dst, uint64_t n, const double *scale,
                               int grid, cudaStream_t st);
cudaError_t launch_spectrum(const SpecArgs &sp, int n_T, cudaStream_t st);

}  // namespace ftk
