// Shared definitions of the FTKomega CUDA path (kernels + host runtime).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define FTK_MAX_SITES 30
#define FTK_MAX_PASS_BONDS 64
#define FTK_MAX_TILE_BITS 16
#define FTK_MAX_RHS 32
#define FTK_MAX_OMEGA 4096
#define FTK_RED_THREADS 256   // threads of the last-block reductions

// One tiled pass of H.v: a CTA owns 2^tile_bits amplitudes whose index bits
// tile_pos[] vary while the bits free_pos[] are fixed by the CTA index.
// Bonds with both sites among tile_pos are applied from shared memory.
// The low chunk_bits tile bits are global bits 0..chunk_bits-1, so a tile is
// a set of contiguous runs of 2^chunk_bits amplitudes (coalesced loads).
struct PassDesc {
    int32_t n_sites;
    int32_t tile_bits;
    int32_t chunk_bits;
    int32_t n_free;
    int32_t first;      // 1: start from zero; 0: add to the partial in out
    int32_t last;       // 1: apply the epilogue
    int32_t n_bonds;
    int32_t pad;
    int32_t tile_pos[FTK_MAX_TILE_BITS];
    int32_t free_pos[FTK_MAX_SITES];
    int32_t bi[FTK_MAX_PASS_BONDS];   // tile-offset bit of site i
    int32_t bj[FTK_MAX_PASS_BONDS];   // tile-offset bit of site j
    // Bond (i, j) of type gamma adds, for parallel (p) / antiparallel (a)
    // spins i, j, the off-diagonal amplitude par/anti to |x ^ 2^i ^ 2^j> and
    // +dg (p) / -dg (a) on the diagonal.
    double par[FTK_MAX_PASS_BONDS];
    double anti[FTK_MAX_PASS_BONDS];
    float par_f[FTK_MAX_PASS_BONDS];    // the same in float for the FP32 kernels
    float anti_f[FTK_MAX_PASS_BONDS];
    float par_lo[FTK_MAX_PASS_BONDS];   // par - par_f, anti - anti_f: low parts of the
    float anti_lo[FTK_MAX_PASS_BONDS];  // double-float kernel's coefficients
    // The diagonal of a pass is dgv[0] c0 + dgv[1] c1 with integer counts
    // c = sum over the pass's bonds of class dgc (+1 parallel, -1 antiparallel):
    // class 0 = x and y bonds (J/4), class 1 = z bonds ((J + K)/4).
    int32_t dgc[FTK_MAX_PASS_BONDS];
    double dgv[2];
    float dgv_f[2];
    float dgv_lo[2];
    // Thread layout of the kernel (filled by hv_layout_pass): a CTA of
    // 2^(tile_bits - le) threads, thread t owns the tile offsets t + 2^tb k
    // for k < 2^le (tb = tile_bits - le), i.e. the top le offset bits are
    // register bits. Bonds are ordered by group: the bonds of group g have
    // the partner-thread mask grp_tmask[g] (the thread bits of their two
    // sites) and occupy [grp_end[g-1], grp_end[g]); the last group has mask 0
    // (partners held by the thread itself, and the diagonal). bcase encodes
    // the register-bit part of the bond mask: 0 none, 1 + a one bit a,
    // 9 + 8a + b two bits a < b.
    int32_t le;
    int32_t cols;      // right-hand sides per launch (column chunk width)
    int32_t n_groups;
    int32_t grp_tmask[FTK_MAX_PASS_BONDS + 1];
    int32_t grp_end[FTK_MAX_PASS_BONDS + 1];
    int8_t bcase[FTK_MAX_PASS_BONDS];
};

namespace ftk {
// double complex as two doubles (16 B, layout of double2)
struct dcx { double re, im; };
}  // namespace ftk

// Device-resident state of the mTPQ iteration (one per context).
struct TpqState {
    double scale;      // s_k = 1 / ||stored psi_k||
    double logQ;       // log Q_k
    double ell;
    double n_sites;
    int32_t k;         // current step
    int32_t pad;
};

// Per-RHS seed-COCG scalars (double), written by the seed kernel.
struct CocgSeed {
    double zs_re, zs_im;        // seed shift
    double e0;                  // shift origin E_j
    double lnorm;               // ||lambda||
    double rho_re, rho_im;      // rho_k = r_k^T r_k
    double rho_prev_re, rho_prev_im;
    double alpha_re, alpha_im;  // alpha_k
    double alpha_prev_re, alpha_prev_im;
    double beta_prev_re, beta_prev_im;  // beta_{k-1}
    double c_re, c_im;          // c_k = beta_{k-1} alpha_k / alpha_{k-1}
    double a1_re, a1_im;        // 1 + c_k - alpha_k z_s: coefficient of r_k in r_{k+1}
    double g_re, g_im;          // g_k = lambda^dagger r_k
    double nrm;                 // ||r_k||
    double resid;               // last max_s ||r_k|| / |pi^s_k| / ||lambda||
    double rescale;             // power of two applied to r_k, r_{k+1}, pi^s in this
                                // iteration (1: none), keeping ||r|| near ||lambda||
    int32_t k;                  // iteration index of this RHS
    int32_t done;               // 1 converged, 2 r^T r vanished, 3 alpha denominator
                                // vanished, 4 max_iter, 5 non-finite residual
    int32_t iters;              // iterations accumulated into G
    int32_t seed_idx;           // shift that is the seed system (moves when the seed switches)
    // Seed switching (the seed converged, shifts remain): this iteration the
    // slowest shift s* became the seed; r_k and w_k are scaled by s1 = 1/pi*_k,
    // r_{k-1} by s0 = 1/pi*_{k-1} (the switch kernel does it), the pi of every
    // shift likewise
    int32_t sw;                 // 1: switched in this iteration
    int32_t switches;           // number of switches so far
    double s1_re, s1_im, s0_re, s0_im;
};

// Dots produced by the vector kernels for each RHS (reduced, double).
// update kernel: [0..1] rho, [2..3] g, [4] |r|^2;  H pass: [0..1] mu
#define FTK_UPD_DOTS 6
#define FTK_HV_DOTS 2
