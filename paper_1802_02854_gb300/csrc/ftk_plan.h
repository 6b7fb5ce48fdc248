// Host-side planner of the tiled H.v passes. Uses no heap memory, so the
// allocation-free entry point can call it too.
#pragma once
#include "ftk_common.cuh"

#include <stdint.h>
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

// Cover of the bonds by tile site sets (greedy, with seeded restarts).
// Every tile keeps the chunk_bits lowest sites (contiguous runs of >= 256 B
// for coalesced loads); the other sites of a pass are added one at a time,
// each time the site that completes the most remaining bonds (ties: the
// site touching most remaining bonds, then a seeded pseudo-random key).
// Restart 0 starts the first pass from the lowest tile_bits sites. The
// cover with the fewest passes (then the largest first pass) is kept.
// Deterministic; uses no heap memory.
struct PlanRng {
    uint32_t s;
    uint32_t next() { s ^= s << 13; s ^= s >> 17; s ^= s << 5; return s; }
};

inline int plan_cover(int n, const PlanBond *bonds, int nb, int b, int c, uint32_t seed, bool low_first,
                      int sets[][FTK_MAX_SITES], int *cnt, int max_passes) {
    char remaining[2 * FTK_MAX_PASS_BONDS];
    int n_rem = nb;
    for (int q = 0; q < nb; ++q) remaining[q] = 1;
    PlanRng rng{seed * 2654435761u + 12345u};
    int np = 0;
    while (n_rem > 0) {
        if (np >= max_passes) return 0;
        char in2[FTK_MAX_SITES];
        memset(in2, 0, sizeof in2);
        int nt = 0;
        int *T = sets[np];
        const int start = (np == 0 && low_first) ? b : c;
        for (int s = 0; s < start; ++s) { T[nt++] = s; in2[s] = 1; }
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
                const long score = (done * 1000 + touch) * 1024 + (seed ? (long)(rng.next() & 1023) : 0);
                if (score > best_score) { best_score = score; best = s; }
            }
            T[nt++] = best;
            in2[best] = 1;
        }
        int taken = 0;
        for (int q = 0; q < nb; ++q)
            if (remaining[q] && in2[bonds[q].i] && in2[bonds[q].j] && taken < FTK_MAX_PASS_BONDS) {
                remaining[q] = 0;
                --n_rem;
                ++taken;
            }
        if (taken == 0) return 0;
        cnt[np++] = taken;
    }
    return np;
}

inline int plan_hv_passes(int n, const PlanBond *bonds, int nb, double K, double J, int elem_bytes,
                          int B, int tile_bits, PassDesc *pd, int max_passes, int *b_out, int *c_out,
                          int restarts = 32) {
    if (n < 2 || n > FTK_MAX_SITES || nb < 1 || nb > 2 * FTK_MAX_PASS_BONDS) return 0;
    int c = 0;
    while (c < n && ((long)1 << c) * B * elem_bytes < 256) ++c;
    int b = tile_bits < n ? tile_bits : n;
    if (b < n && c > b - 2) c = b - 2 > 0 ? b - 2 : 0;   // later passes need >= 2 free tile bits
    if (c > b) c = b;
    *b_out = b;
    *c_out = c;
    if (max_passes > FTK_MAX_PASSES) max_passes = FTK_MAX_PASSES;
    int best_sets[FTK_MAX_PASSES][FTK_MAX_SITES], best_cnt[FTK_MAX_PASSES];
    int best_np = 0;
    for (int r = 0; r <= restarts; ++r) {
        int sets[FTK_MAX_PASSES][FTK_MAX_SITES], cnt[FTK_MAX_PASSES];
        const int np = plan_cover(n, bonds, nb, b, c, (uint32_t)r, r == 0, sets, cnt, max_passes);
        if (np > 0 && (best_np == 0 || np < best_np || (np == best_np && cnt[0] > best_cnt[0]))) {
            best_np = np;
            memcpy(best_sets, sets, sizeof sets);
            memcpy(best_cnt, cnt, sizeof cnt);
        }
        if (b >= n) break;
    }
    if (best_np == 0) return 0;
    // materialise the passes: each bond goes to the first pass containing it
    char remaining[2 * FTK_MAX_PASS_BONDS];
    for (int q = 0; q < nb; ++q) remaining[q] = 1;
    int np = 0;
    for (int k = 0; k < best_np; ++k) {
        int T[FTK_MAX_SITES];
        for (int s = 0; s < b; ++s) T[s] = best_sets[k][s];
        for (int a = 1; a < b; ++a)   // ascending: chunk sites first
            for (int m = a; m > 0 && T[m - 1] > T[m]; --m) { const int t = T[m]; T[m] = T[m - 1]; T[m - 1] = t; }
        char in_t[FTK_MAX_SITES];
        memset(in_t, 0, sizeof in_t);
        for (int s = 0; s < b; ++s) in_t[T[s]] = 1;
        PassDesc &p = pd[np];
        memset(&p, 0, sizeof p);
        p.n_sites = n;
        p.tile_bits = b;
        p.chunk_bits = c;
        p.n_free = n - b;
        int tpos[FTK_MAX_SITES];
        for (int s = 0; s < n; ++s) tpos[s] = -1;
        for (int s = 0; s < b; ++s) { p.tile_pos[s] = T[s]; tpos[T[s]] = s; }
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
            p.par_lo[taken] = (float)(par - (double)p.par_f[taken]);
            p.anti_lo[taken] = (float)(anti - (double)p.anti_f[taken]);
            p.dgc[taken] = bonds[q].g == 2 ? 1 : 0;
            remaining[q] = 0;
            ++taken;
        }
        if (taken == 0) continue;
        p.n_bonds = taken;
        p.dgv[0] = J / 4;
        p.dgv[1] = (J + K) / 4;
        p.dgv_f[0] = (float)p.dgv[0];
        p.dgv_f[1] = (float)p.dgv[1];
        p.dgv_lo[0] = (float)(p.dgv[0] - (double)p.dgv_f[0]);
        p.dgv_lo[1] = (float)(p.dgv[1] - (double)p.dgv_f[1]);
        ++np;
    }
    for (int q = 0; q < nb; ++q)
        if (remaining[q]) return 0;
    for (int k = 0; k < np; ++k) {
        pd[k].first = k == 0;
        pd[k].last = k == np - 1;
    }
    return np;
}

// Site relabelling for fewer H.v passes. The chunk sites (the lowest index
// bits, fixed by the memory layout) sit in every tile, so which sites carry
// the lowest labels matters. Tries `trials` seeded choices of the chunk sites
// (and the given labelling) and returns in perm (site l -> new label
// perm[l]) the labelling whose plan has the fewest passes; returns that
// number of passes (0 on failure).
inline int plan_suggest_order(int n, const PlanBond *bonds, int nb, int elem_bytes, int B, int tile_bits, int *perm,
                              int trials = 64) {
    PassDesc pd[FTK_MAX_PASSES];
    int b = 0, c = 0;
    for (int s = 0; s < n; ++s) perm[s] = s;
    int best = plan_hv_passes(n, bonds, nb, -1.0, 0.1, elem_bytes, B, tile_bits, pd, FTK_MAX_PASSES, &b, &c, 16);
    if (best == 0) return 0;
    PlanRng rng{0x9e3779b9u};
    for (int t = 0; t < trials && best > 1; ++t) {
        int cand[FTK_MAX_SITES];
        char used[FTK_MAX_SITES];
        memset(used, 0, sizeof used);
        int next = 0;
        for (int k = 0; k < c; ++k) {
            int s;
            do { s = (int)(rng.next() % (uint32_t)n); } while (used[s]);
            used[s] = 1;
            cand[s] = next++;
        }
        for (int s = 0; s < n; ++s)
            if (!used[s]) cand[s] = next++;
        PlanBond rb[2 * FTK_MAX_PASS_BONDS];
        for (int q = 0; q < nb; ++q) rb[q] = {cand[bonds[q].i], cand[bonds[q].j], bonds[q].g};
        const int np = plan_hv_passes(n, rb, nb, -1.0, 0.1, elem_bytes, B, tile_bits, pd, FTK_MAX_PASSES, &b, &c, 16);
        if (np > 0 && np < best) {
            best = np;
            for (int s = 0; s < n; ++s) perm[s] = cand[s];
        }
    }
    return best;
}

}  // namespace ftk
