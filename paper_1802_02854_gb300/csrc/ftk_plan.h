// Host-side planner of the tiled H.v passes. Uses no heap memory, so the
// allocation-free entry point can call it too.
#pragma once
#include "ftk_common.cuh"

#include <math.h>
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

// Local search for a cover with np passes: every pass holds the chunk sites
// and b - c other sites. The chunk sites are the lowest c labels, or, with
// joint_chunk, any c sites (searched too; returned in chunk_out). Simulated
// annealing on the number of bonds whose two sites share a pass: seeded,
// at most `steps` moves, no heap memory. On success (every bond covered)
// sets[p] holds the b sites of pass p, chunk sites first.
inline bool plan_anneal_cover(int n, const PlanBond *bonds, int nb, int b, int c, int np, uint32_t seed,
                              long steps, bool joint_chunk, int sets[][FTK_MAX_SITES], int *chunk_out) {
    if (np < 1 || np > FTK_MAX_PASSES || b >= n || c > b || c < 0) return false;
    const int m = b - c;   // non-chunk sites per pass
    if (m < 1) return false;
    PlanRng rng{seed * 2654435761u + 0x9e3779b9u};
    if (rng.s == 0) rng.s = 1;
    char chunk[FTK_MAX_SITES];
    char mem[FTK_MAX_PASSES][FTK_MAX_SITES];
    memset(chunk, 0, sizeof chunk);
    memset(mem, 0, sizeof mem);
    // a uniformly drawn site with flag test() true (bounded rejection sampling)
    auto draw = [&](auto test) -> int {
        for (int t = 0; t < 4096; ++t) {
            const int s = (int)(rng.next() % (uint32_t)n);
            if (test(s)) return s;
        }
        for (int s = 0; s < n; ++s)
            if (test(s)) return s;
        return -1;
    };
    if (!joint_chunk) {
        for (int s = 0; s < c; ++s) chunk[s] = 1;
    } else {
        for (int k = 0; k < c; ++k) chunk[draw([&](int s) { return !chunk[s]; })] = 1;
    }
    for (int p = 0; p < np; ++p)
        for (int k = 0; k < m; ++k) mem[p][draw([&](int s) { return !chunk[s] && !mem[p][s]; })] = 1;
    auto covered = [&]() {
        int cov = 0;
        for (int q = 0; q < nb; ++q) {
            const int i = bonds[q].i, j = bonds[q].j;
            for (int p = 0; p < np; ++p)
                if ((chunk[i] || mem[p][i]) && (chunk[j] || mem[p][j])) { ++cov; break; }
        }
        return cov;
    };
    int cur = covered();
    double T = 2.0;
    for (long st = 0; st < steps && cur < nb; ++st) {
        int kind, p = 0, a = -1, x = -1;
        char moved[FTK_MAX_PASSES];
        if (joint_chunk && c > 0 && rng.next() % 10 == 0) {
            // a chunk site and a non-chunk site trade places (in every pass
            // that held x, a takes its place)
            kind = 0;
            a = draw([&](int s) { return chunk[s] != 0; });
            x = draw([&](int s) { return !chunk[s]; });
            chunk[a] = 0;
            chunk[x] = 1;
            for (int q = 0; q < np; ++q) {
                moved[q] = mem[q][x];
                if (moved[q]) { mem[q][x] = 0; mem[q][a] = 1; }
            }
        } else {
            // pass p swaps one of its sites for another
            kind = 1;
            p = (int)(rng.next() % (uint32_t)np);
            a = draw([&](int s) { return mem[p][s] != 0; });
            x = draw([&](int s) { return !chunk[s] && !mem[p][s]; });
            mem[p][a] = 0;
            mem[p][x] = 1;
        }
        const int nw = covered();
        const double u = (double)(rng.next() >> 8) * (1.0 / 16777216.0);
        if (nw >= cur || u < exp((nw - cur) / T)) {
            cur = nw;
        } else if (kind == 0) {
            chunk[x] = 0;
            chunk[a] = 1;
            for (int q = 0; q < np; ++q)
                if (moved[q]) { mem[q][a] = 0; mem[q][x] = 1; }
        } else {
            mem[p][x] = 0;
            mem[p][a] = 1;
        }
        T = T * 0.9995 > 0.05 ? T * 0.9995 : 0.05;
    }
    if (cur < nb) return false;
    int k = 0;
    for (int s = 0; s < n; ++s)
        if (chunk[s]) { if (chunk_out) chunk_out[k] = s; ++k; }
    for (int p = 0; p < np; ++p) {
        int t = 0;
        for (int s = 0; s < n; ++s)
            if (chunk[s]) sets[p][t++] = s;
        for (int s = 0; s < n; ++s)
            if (mem[p][s]) sets[p][t++] = s;
    }
    return true;
}

// Moves of one local-search restart (context plans and site relabelling; the
// allocation-free entry point plans greedily only).
constexpr long kPlanLocalSteps = 30000;

// local_steps > 0: after the greedy covers, a local search (plan_anneal_cover,
// 8 seeded restarts of local_steps moves) looks for covers with fewer passes.
inline int plan_hv_passes(int n, const PlanBond *bonds, int nb, double K, double J, int elem_bytes,
                          int B, int tile_bits, PassDesc *pd, int max_passes, int *b_out, int *c_out,
                          int restarts = 32, long local_steps = 0) {
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
    if (local_steps > 0 && b < n) {
        for (int target = best_np - 1; target >= 1; --target) {
            bool found = false;
            for (int r = 0; r < 8 && !found; ++r) {
                int sets[FTK_MAX_PASSES][FTK_MAX_SITES];
                if (plan_anneal_cover(n, bonds, nb, b, c, target, 1000u + (uint32_t)r, local_steps, false, sets,
                                      nullptr)) {
                    memcpy(best_sets, sets, sizeof sets);
                    best_np = target;
                    found = true;
                }
            }
            if (!found) break;
        }
    }
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
    // local search over the chunk sites and the passes together; a cover with
    // fewer passes fixes the chunk sites (lowest labels, the other sites in
    // their order after them), kept if the planner with its own local search
    // reaches that count on the relabelled bonds
    for (int target = best - 1; b < n && target >= 1; --target) {
        bool found = false;
        for (int r = 0; r < 8 && !found; ++r) {
            int sets[FTK_MAX_PASSES][FTK_MAX_SITES], chunk[FTK_MAX_SITES];
            if (!plan_anneal_cover(n, bonds, nb, b, c, target, 7u + (uint32_t)r, kPlanLocalSteps, true, sets, chunk))
                continue;
            int cand[FTK_MAX_SITES];
            char is_chunk[FTK_MAX_SITES];
            memset(is_chunk, 0, sizeof is_chunk);
            for (int k = 0; k < c; ++k) { cand[chunk[k]] = k; is_chunk[chunk[k]] = 1; }
            int next = c;
            for (int s = 0; s < n; ++s)
                if (!is_chunk[s]) cand[s] = next++;
            PlanBond rb[2 * FTK_MAX_PASS_BONDS];
            for (int q = 0; q < nb; ++q) rb[q] = {cand[bonds[q].i], cand[bonds[q].j], bonds[q].g};
            const int np = plan_hv_passes(n, rb, nb, -1.0, 0.1, elem_bytes, B, tile_bits, pd, FTK_MAX_PASSES, &b, &c,
                                          16, kPlanLocalSteps);
            if (np > 0 && np <= target) {
                best = np;
                for (int s = 0; s < n; ++s) perm[s] = cand[s];
                found = true;
            }
        }
        if (!found) break;
    }
    return best;
}

}  // namespace ftk
