// Host-side planner of the tiled H.v passes. Uses no heap memory, so the
// allocation-free entry point can call it too.
#pragma once
#include "ftk_common.cuh"

#include <string.h>

#define FTK_MAX_PASSES 16

namespace ftk {

struct PlanBond { int i, j, g; };

// Matrix elements of h_b = J S_i.S_j + K S^g_i S^g_j on the S^z basis:
//   S^x S^x |x> = 1/4 |x'>, S^y S^y |x> = -s_i s_j / 4 |x'>, S^z S^z = s_i s_j / 4
// with x' = x ^ 2^i ^ 2^j, so for parallel (p) / antiparallel (a) spins
//   x-bond: p K/4,  a K/4 + J/2;  y-bond: p -K/4, a K/4 + J/2;  z-bond: p 0, a J/2
// and the diagonal is +dg (p) / -dg (a) with dg = J/4 (x, y), (J + K)/4 (z).
inline void bond_coefficients(int g, double K, double J, double *par, double *anti) {
    if (g == 0) { *par = K / 4; *anti = K / 4 + J / 2; }
    else if (g == 1) { *par = -K / 4; *anti = K / 4 + J / 2; }
    else { *par = 0; *anti = J / 2; }
}

// Greedy cover of the bonds by tile bit sets. The first pass takes the low
// tile_bits sites (good when neighbouring sites have close labels); each
// later pass keeps the chunk_bits lowest sites (contiguous runs of >= 256 B
// for coalesced loads) and adds, one at a time, the site that completes the
// most remaining bonds. Returns the number of passes (0 on failure).
inline int plan_hv_passes(int n, const PlanBond *bonds, int nb, double K, double J, int elem_bytes,
                          int B, int tile_bits, PassDesc *pd, int max_passes, int *b_out, int *c_out) {
    if (n < 2 || n > FTK_MAX_SITES || nb < 1 || nb > 2 * FTK_MAX_PASS_BONDS) return 0;
    int c = 0;
    while (c < n && ((long)1 << c) * B * elem_bytes < 256) ++c;
    int b = tile_bits < n ? tile_bits : n;
    if (b < n && c > b - 2) c = b - 2 > 0 ? b - 2 : 0;   // later passes need >= 2 free tile bits
    if (c > b) c = b;
    *b_out = b;
    *c_out = c;
    char remaining[2 * FTK_MAX_PASS_BONDS];
    int n_rem = nb;
    for (int q = 0; q < nb; ++q) remaining[q] = 1;
    int T[FTK_MAX_SITES];
    int nt = 0;
    for (int s = 0; s < b; ++s) T[nt++] = s;
    int np = 0;
    while (n_rem > 0) {
        if (np >= max_passes) return 0;
        char in_t[FTK_MAX_SITES];
        memset(in_t, 0, sizeof in_t);
        for (int k = 0; k < nt; ++k) in_t[T[k]] = 1;
        // sort T ascending (chunk bits first)
        for (int a = 1; a < nt; ++a)
            for (int k = a; k > 0 && T[k - 1] > T[k]; --k) { int t = T[k]; T[k] = T[k - 1]; T[k - 1] = t; }
        PassDesc &p = pd[np];
        memset(&p, 0, sizeof p);
        p.n_sites = n;
        p.tile_bits = b;
        p.chunk_bits = c;
        p.n_free = n - b;
        int tpos[FTK_MAX_SITES];
        for (int s = 0; s < n; ++s) tpos[s] = -1;
        for (int k = 0; k < b; ++k) { p.tile_pos[k] = T[k]; tpos[T[k]] = k; }
        int f = 0;
        for (int s = 0; s < n; ++s)
            if (!in_t[s]) p.free_pos[f++] = s;
        int taken = 0;
        for (int q = 0; q < nb && taken < FTK_MAX_PASS_BONDS; ++q) {
            if (!remaining[q] || !in_t[bonds[q].i] || !in_t[bonds[q].j]) continue;
            double par, anti;
            bond_coefficients(bonds[q].g, K, J, &par, &anti);
            p.bi[taken] = tpos[bonds[q].i];
            p.bj[taken] = tpos[bonds[q].j];
            p.par[taken] = par;
            p.anti[taken] = anti;
            p.par_f[taken] = (float)par;
            p.anti_f[taken] = (float)anti;
            p.dgc[taken] = bonds[q].g == 2 ? 1 : 0;
            remaining[q] = 0;
            --n_rem;
            ++taken;
        }
        if (taken == 0) return 0;
        p.n_bonds = taken;
        p.dgv[0] = J / 4;
        p.dgv[1] = (J + K) / 4;
        p.dgv_f[0] = (float)p.dgv[0];
        p.dgv_f[1] = (float)p.dgv[1];
        ++np;
        if (n_rem == 0) break;
        // next tile set: chunk bits plus greedily chosen sites
        char in2[FTK_MAX_SITES];
        memset(in2, 0, sizeof in2);
        nt = 0;
        for (int s = 0; s < c; ++s) { T[nt++] = s; in2[s] = 1; }
        while (nt < b) {
            int best = -1;
            long best_score = -1;
            for (int s = 0; s < n; ++s) {
                if (in2[s]) continue;
                long done = 0, touch = 0;
                for (int q = 0; q < nb; ++q) {
                    if (!remaining[q] || (bonds[q].i != s && bonds[q].j != s)) continue;
                    ++touch;
                    const int other = bonds[q].i == s ? bonds[q].j : bonds[q].i;
                    if (in2[other]) ++done;
                }
                const long score = done * 1000 + touch;
                if (score > best_score) { best_score = score; best = s; }
            }
            T[nt++] = best;
            in2[best] = 1;
        }
    }
    for (int k = 0; k < np; ++k) {
        pd[k].first = k == 0;
        pd[k].last = k == np - 1;
    }
    return np;
}

}  // namespace ftk
