// One tiled pass of the matrix-free Kitaev-Heisenberg H.V on sm_103a (Sec.
// IV.A: every method of the paper is costed in these products), with fused
// epilogues for the mTPQ step (Appendix A) and the COCG mu = r^T H r dot.
//
// Data: B right-hand sides stored one after the other, element (x, j) at
// j * ld + x (ld = 2^N). A CTA owns tiles of 2^b amplitudes: the offset bits of a tile
// are the global bits pd.tile_pos[], the other bits (pd.free_pos[]) are fixed
// by the tile index; the low offset bits are global bits 0..chunk-1 so every
// tile is a set of >= 256-byte contiguous runs. Persistent CTAs loop over
// tiles; the next tile is fetched with cp.async into the second of two
// shared-memory buffers while the current one is processed, and the partial
// product of earlier passes is prefetched into a third.
//
// Thread layout: T = 2^tb threads, thread t owns the offsets o = t + T k,
// k < E = 2^le (register bits = the top le offset bits), with accumulators
// for all E x B amplitudes in registers. A bond (i, j) has partner o ^ m,
// m = 2^bi | 2^bj: its thread part selects the partner thread t ^ tm, its
// register part the partner register k ^ km. Bonds with the same tm form a
// group: the thread reads the partner thread's E x B amplitudes once from
// shared memory and applies every bond of the group from registers (the
// coefficient choice par/anti is resolved once per thread and bond from the
// thread bits, and at compile time from the register bits). The group with
// tm = 0 holds the bonds between register sites, and the diagonal.
//
// Two kernels: hv_pass_kernel (FP64 / FP32 amplitudes, several columns per
// launch) and hv_pass_df_kernel (double-float amplitudes, hi + lo float
// pairs, one column per launch; a tile amplitude's hi and lo parts side by
// side in one float4; a variant with the tile stride as a compile-time
// constant; a variant whose first pass also performs the COCG residual update
// of the previous step).
#include "ftk_common.cuh"
#include "ftk_device.cuh"
#include "ftk_kernels.h"

#include <algorithm>
#include <mutex>
#include <type_traits>

namespace ftk {

// ------------------------------------------------------------ async copies
// L2 prefetch of the 128-byte line holding p (no register result)
__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
__device__ __forceinline__ void cp_async_elem(float2 *dst, const float2 *src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_elem(double2 *dst, const double2 *src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// -------------------------------------------------------- bond application
template <int KA, int KB>
struct KMask {
    static constexpr int m = (KA >= 0 ? (1 << KA) : 0) | (KB >= 0 ? (1 << KB) : 0);
};

// acc += c p for a complex amplitude and a real coefficient: on sm_100 and
// later, float pairs take one packed FMA (fma.rn.f32x2) for both components
__device__ __forceinline__ void cfma(double c, const double2 &p, double2 &acc) {
    acc.x = fma(c, p.x, acc.x);
    acc.y = fma(c, p.y, acc.y);
}
__device__ __forceinline__ void cfma(float c, const float2 &p, float2 &acc) {
    acc = __ffma2_rn(make_float2(c, c), p, acc);
}
__device__ __forceinline__ void cadd(const double2 &p, double2 &acc) { acc.x += p.x; acc.y += p.y; }
__device__ __forceinline__ void cadd(const float2 &p, float2 &acc) { acc = __fadd2_rn(acc, p); }

// acc[k] += c(k) P[k ^ km]: c = cs where the register bits of the bond are
// parallel (k-parity 0), cf otherwise; k, k ^ km and the choice are
// compile-time after unrolling.
template <typename R, int B, int LE, int KA, int KB>
__device__ __forceinline__ void bond_apply(typename C2<R>::t (&acc)[1 << LE][B], const typename C2<R>::t (&pv)[1 << LE][B],
                                           R cs, R cf) {
    constexpr int E = 1 << LE;
#pragma unroll
    for (int k = 0; k < E; ++k) {
        const int kpar = (KA >= 0 ? (k >> KA) & 1 : 0) ^ (KB >= 0 ? (k >> KB) & 1 : 0);
        const int kp = k ^ KMask<KA, KB>::m;
        const R c = kpar ? cf : cs;
#pragma unroll
        for (int j = 0; j < B; ++j) cfma(c, pv[kp][j], acc[k][j]);
    }
}

#define FTK_HV_CASE(ID, KA, KB)                                                             \
    case ID:                                                                                \
        if constexpr (KA < LE && KB < LE) bond_apply<R, B, LE, KA, KB>(acc, pv, cs, cf);    \
        break;

// TB > 0: the thread bits of the tile (tile_bits - LE) as a compile-time
// constant, so that the strides T k of the shared tile fold into immediate
// offsets (one vector with 512 threads: the 2^13-amplitude FP32 and
// 2^12-amplitude FP64 tiles, TB = 9).
template <typename R, int B, int LE, int EPI, int TB = 0>
__global__ void __launch_bounds__(512, 1)
hv_pass_kernel(const typename C2<R>::t *__restrict__ in, typename C2<R>::t *out, long long ld, const PassDesc pd,
               const EpiArgs ea) {
    typedef typename C2<R>::t cx;
    constexpr int E = 1 << LE;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (ea.all_done && *ea.all_done) return;
    if (ea.lowp && *ea.lowp != ea.lowp_run) return;
    const int b = TB > 0 ? TB + LE : pd.tile_bits;
    const int tb = b - LE;
    const int tile_n = 1 << b;
    const int T = 1 << tb;
    const int t = threadIdx.x;
    const bool act = t < T;
    cx *buf0 = reinterpret_cast<cx *>(smem_raw);
    cx *buf1 = buf0 + (size_t)tile_n * B;
    cx *pbuf = buf1 + (size_t)tile_n * B;   // partial product of earlier passes
    double *red = reinterpret_cast<double *>(pbuf + (size_t)tile_n * B);

    // element offset of (offset t + T k, column j) from the tile base:
    // st + ksp(k) + j ld, with st / ksp the global bits of the thread /
    // register part (disjoint bits, so OR = sum)
    // (32-bit: a column has at most 2^FTK_MAX_SITES elements)
    uint32_t st = 0;
    for (int q = 0; q < tb; ++q)
        if ((t >> q) & 1) st |= 1u << pd.tile_pos[q];
    uint32_t kofs[LE > 0 ? LE : 1];
#pragma unroll
    for (int q = 0; q < LE; ++q) kofs[q] = 1u << pd.tile_pos[tb + q];
    auto eofs = [&](int k) -> uint32_t {
        uint32_t v = st;
#pragma unroll
        for (int q = 0; q < LE; ++q)
            if ((k >> q) & 1) v += kofs[q];
        return v;
    };
    // tile offsets: the bits of the tile index deposited at the free sites.
    // Successive tiles of a CTA are gridDim.x apart; their offsets follow by
    // a masked addition (the bits outside the mask set to 1 carry across
    // them): dep(a + g) = ((dep(a) | ~mask) + dep(g)) & mask.
    auto tile_ofs = [&](long tau) -> long long {
        uint64_t v = 0;
        for (int q = 0; q < pd.n_free; ++q)
            if ((tau >> q) & 1) v |= 1ull << pd.free_pos[q];
        return (long long)v;
    };
    // (mask and step in shared memory: read once per tile, no registers held)
    __shared__ uint64_t free_mask, dep_grid;
    if (threadIdx.x == 0) {
        uint64_t m = 0;
        for (int q = 0; q < pd.n_free; ++q) m |= 1ull << pd.free_pos[q];
        free_mask = m;
        dep_grid = (uint64_t)tile_ofs(gridDim.x);
    }
    __syncthreads();
    auto next_ofs = [&](long long ofs) -> long long {
        const uint64_t m = free_mask;
        return (long long)((((uint64_t)ofs | ~m) + dep_grid) & m);
    };
    // diagonal of this pass's bonds at the thread's offsets: dgv[0] c0 +
    // dgv[1] c1 with integer counts c (+1 parallel, -1 antiparallel; parity
    // = thread part ^ register part), two multiply-adds per amplitude
    R dg[E];
    {
        int c0[E], c1[E];
#pragma unroll
        for (int k = 0; k < E; ++k) { c0[k] = 0; c1[k] = 0; }
        for (int l = 0; l < pd.n_bonds; ++l) {
            const int m = (1 << pd.bi[l]) | (1 << pd.bj[l]);
            const int pt = __popc(t & m & (T - 1)) & 1;
            const int km = m >> tb;
            const int cls = pd.dgc[l];
#pragma unroll
            for (int k = 0; k < E; ++k) {
                const int sg = 1 - 2 * ((pt ^ __popc(k & km)) & 1);
                c0[k] += cls ? 0 : sg;
                c1[k] += cls ? sg : 0;
            }
        }
        const R d0 = Coef<R>::dgv(pd, 0), d1 = Coef<R>::dgv(pd, 1);
#pragma unroll
        for (int k = 0; k < E; ++k) dg[k] = (R)c0[k] * d0 + (R)c1[k] * d1;
    }
    const R scale = (EPI == EPI_TPQ) ? (R)(*ea.scale) : (R)1;
    const R ell = (R)ea.ell, inv_n = (R)ea.inv_n;
    // EPI_COCG_MIXED: the mixed mode's COCG epilogue; its input is the hi part
    // of a float hi + lo residual and mu is accumulated from hi + lo with
    // exact FMA two-products and two-sums (double-float, ~48 bits) on the
    // FP32 pipe
    constexpr bool MIX = EPI == EPI_COCG_MIXED;
    constexpr int ND = (EPI == EPI_TPQ || EPI == EPI_TAYLOR) ? 2 : ((EPI == EPI_COCG || MIX) ? 2 * B : 1);
    const R tcoef = (EPI == EPI_TAYLOR) ? (R)ea.tcoef : (R)0;
    Acc<R> dot[ND];
    const bool first = pd.first != 0;

    // async copy of a tile of `src` (the thread's own elements) into buf
    auto issue = [&](const cx *src, long long tofs, cx *buf) {
        if (act) {
            const cx *g = src + tofs;
#pragma unroll
            for (int k = 0; k < E; ++k) {
                const cx *gk = g + eofs(k);
#pragma unroll
                for (int j = 0; j < B; ++j) cp_async_elem(buf + (size_t)j * tile_n + t + T * k, gk + (size_t)j * ld);
            }
        }
        cp_async_commit();
    };
    // Pipeline (commit order): v_0 [p_0] | per tile i: v_{i+1}, then after
    // tile i's epilogue p_{i+1}. Each thread reads back only the partial
    // elements it copied itself, so pbuf needs no block barrier.
    const long n_tiles = 1L << pd.n_free;
    long tau = blockIdx.x;
    long long tofs = tau < n_tiles ? tile_ofs(tau) : 0;
    if (tau < n_tiles) {
        issue(in, tofs, buf0);
        if (!first) issue(out, tofs, pbuf);
    }
    for (int it = 0; tau < n_tiles; tau += gridDim.x, ++it) {
        const cx *cur = (it & 1) ? buf1 : buf0;
        cx *nxt = (it & 1) ? buf0 : buf1;
        const long tn = tau + gridDim.x;
        const bool more = tn < n_tiles;
        const long long tofs_n = more ? next_ofs(tofs) : 0;
        if (more) issue(in, tofs_n, nxt);
        // v of this tile: everything but the newest one (first pass) or two groups
        if (first) { if (more) cp_async_wait<1>(); else cp_async_wait<0>(); }
        else { if (more) cp_async_wait<2>(); else cp_async_wait<1>(); }
        __syncthreads();
        if (act) {
            cx acc[E][B];   // (re, im) accumulators
            cx pv[E][B];    // partner amplitudes of the current group
#pragma unroll
            for (int k = 0; k < E; ++k)
#pragma unroll
                for (int j = 0; j < B; ++j) acc[k][j] = mk<R>((R)0, (R)0);
            int q = 0;
            for (int g = 0; g < pd.n_groups; ++g) {
                const int tm = pd.grp_tmask[g];
                const cx *src = cur + (t ^ tm);
#pragma unroll
                for (int k = 0; k < E; ++k)
#pragma unroll
                    for (int j = 0; j < B; ++j) pv[k][j] = src[(size_t)j * tile_n + T * k];
                const int pt = __popc(t & tm) & 1;
                for (const int end = pd.grp_end[g]; q < end; ++q) {
                    const R par = Coef<R>::par(pd, q), anti = Coef<R>::anti(pd, q);
                    const R cs = pt ? anti : par, cf = pt ? par : anti;
                    switch (pd.bcase[q]) {
                        FTK_HV_CASE(0, -1, -1)
                        FTK_HV_CASE(1, 0, -1)
                        FTK_HV_CASE(2, 1, -1)
                        FTK_HV_CASE(3, 2, -1)
                        FTK_HV_CASE(4, 3, -1)
                        FTK_HV_CASE(5, 4, -1)
                        FTK_HV_CASE(10, 0, 1)
                        FTK_HV_CASE(11, 0, 2)
                        FTK_HV_CASE(12, 0, 3)
                        FTK_HV_CASE(13, 0, 4)
                        FTK_HV_CASE(19, 1, 2)
                        FTK_HV_CASE(20, 1, 3)
                        FTK_HV_CASE(21, 1, 4)
                        FTK_HV_CASE(28, 2, 3)
                        FTK_HV_CASE(29, 2, 4)
                        FTK_HV_CASE(37, 3, 4)
                        default: break;
                    }
                }
            }
            // the last group is the thread's own amplitudes: diagonal
#pragma unroll
            for (int k = 0; k < E; ++k)
#pragma unroll
                for (int j = 0; j < B; ++j) cfma(dg[k], pv[k][j], acc[k][j]);
            if (!first) {   // partial product of the earlier passes (own elements)
                if (more) cp_async_wait<1>(); else cp_async_wait<0>();
#pragma unroll
                for (int k = 0; k < E; ++k)
#pragma unroll
                    for (int j = 0; j < B; ++j) cadd(pbuf[(size_t)j * tile_n + t + T * k], acc[k][j]);
            }
            cx *o = out + tofs;
#pragma unroll
            for (int k = 0; k < E; ++k) {
                cx *ok = o + eofs(k);
                if (!pd.last || EPI == EPI_PLAIN) {
#pragma unroll
                    for (int j = 0; j < B; ++j) ok[(size_t)j * ld] = acc[k][j];
                } else if constexpr (EPI == EPI_TPQ) {
                    // psi' = s (l v - H v / N);  <v|Hv>, |psi'|^2
                    const R yr = scale * (ell * pv[k][0].x - inv_n * acc[k][0].x);
                    const R yi = scale * (ell * pv[k][0].y - inv_n * acc[k][0].y);
                    ok[0] = mk<R>(yr, yi);
                    dot[0].fma2(pv[k][0].x, acc[k][0].x);
                    dot[0].fma2(pv[k][0].y, acc[k][0].y);
                    dot[1].fma2(yr, yr);
                    dot[1].fma2(yi, yi);
                } else if constexpr (EPI == EPI_TAYLOR) {
                    // cTPQ Taylor term: t' = c (l v - H v / N), acc += t';
                    // <v|Hv> (the energy of v), |acc|^2
                    const R yr = tcoef * (ell * pv[k][0].x - inv_n * acc[k][0].x);
                    const R yi = tcoef * (ell * pv[k][0].y - inv_n * acc[k][0].y);
                    ok[0] = mk<R>(yr, yi);
                    cx *ap = reinterpret_cast<cx *>(ea.taylor_acc) + tofs + eofs(k);
                    cx a = *ap;
                    a.x += yr;
                    a.y += yi;
                    *ap = a;
                    dot[0].fma2(pv[k][0].x, acc[k][0].x);
                    dot[0].fma2(pv[k][0].y, acc[k][0].y);
                    dot[1].fma2(a.x, a.x);
                    dot[1].fma2(a.y, a.y);
                } else if constexpr (EPI == EPI_COCG) {
                    // W = H R;  mu_j = R_j^T W_j (bilinear)
#pragma unroll
                    for (int j = 0; j < B; ++j) {
                        ok[(size_t)j * ld] = acc[k][j];
                        dot[2 * j].fma2(pv[k][j].x, acc[k][j].x);
                        dot[2 * j].fma2(-pv[k][j].y, acc[k][j].y);
                        dot[2 * j + 1].fma2(pv[k][j].x, acc[k][j].y);
                        dot[2 * j + 1].fma2(pv[k][j].y, acc[k][j].x);
                    }
                } else if constexpr (MIX) {
                    // mixed mode: R = hi + lo, mu_j = R_j^T W_j in double-float
#pragma unroll
                    for (int j = 0; j < B; ++j) {
                        ok[(size_t)j * ld] = acc[k][j];
                        const float2 lo =
                            reinterpret_cast<const float2 *>(ea.lo)[tofs + eofs(k) + (size_t)j * ld];
                        dot[2 * j].fma_hl(pv[k][j].x, lo.x, acc[k][j].x);
                        dot[2 * j].fma_hl(-pv[k][j].y, -lo.y, acc[k][j].y);
                        dot[2 * j + 1].fma_hl(pv[k][j].x, lo.x, acc[k][j].y);
                        dot[2 * j + 1].fma_hl(pv[k][j].y, lo.y, acc[k][j].x);
                    }
                }
            }
        }
        if (!first && more) issue(out, tofs_n, pbuf);
        tofs = tofs_n;
        __syncthreads();   // buffer `cur` is refilled two tiles later
    }
    cp_async_wait<0>();
    if (EPI == EPI_PLAIN || !pd.last) return;

    double v[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) v[d] = dot[d].get();
    block_reduce<ND>(v, red);
    if (threadIdx.x < ND) ea.partials[(size_t)blockIdx.x * ND + threadIdx.x] = red[threadIdx.x];
    double *res = ea.result;
    if (!last_block_reduce<ND>(ea.partials, ea.counter, res, red)) return;
    if (EPI == EPI_TPQ && threadIdx.x == 0) {
        // mTPQ statistics of step k (Appendix A): u_k = s^2 <v|Hv>/N,
        // q_k = ||psi'||, <H^2>_k = N^2 (q^2 - l^2 + 2 l u_k)
        TpqState *stt = ea.tpq;
        const double s = stt->scale, n = stt->n_sites, l = stt->ell;
        const double u = s * s * res[0] / n;
        const double q2 = res[1];
        const int k = stt->k;
        ea.stat_u[k] = u;
        ea.stat_logq[k] = stt->logQ;
        ea.stat_h2[k] = n * n * (q2 - l * l + 2.0 * l * u);
        stt->logQ += 0.5 * log(q2);
        stt->scale = 1.0 / sqrt(q2);
        stt->k = k + 1;
    }
}

// ------------------------------------------------------------------------
// Double-float H.V (precision mode FTK_DF): FP64-class accuracy on the FP32
// pipe, which on GB300 issues 64x the FP64 rate. A vector is a pair of float
// arrays, hi and lo (lo df_lo float2 elements after hi), value hi + lo
// (~48 significant bits). The tile holds an amplitude's hi and lo parts
// together (one float4); a bond adds c * p with the exact FMA two-product of the hi parts,
// the cross terms, and Knuth's two-sum into an accumulator (hi, lo) whose lo
// part collects the rounding errors (renormalised when stored). One column
// per launch, E = 2^LE amplitudes per thread, same tiling, groups and
// pipeline as the kernel above.
// The real and imaginary components take the same operations with the same
// coefficient, so every step runs on float pairs (re, im) as one packed
// f32x2 instruction (sm_100 and later). No step negates an operand: a - b is
// formed as fma(b, -1, a) (the same rounding as the subtraction) and the
// product's error term from the negated coefficient -c_hi, so each complex
// term costs 12 packed instructions. h, l: the (re, im) hi and lo parts of
// the accumulator.
__device__ __forceinline__ float2 m1x2() { return make_float2(-1.f, -1.f); }
__device__ __forceinline__ float2 fsub2(float2 a, float2 b) { return __ffma2_rn(b, m1x2(), a); }   // a - b
// acc += c p, c = ch + cl, p = ph + pl; nch = -ch, ncl = -cl:
//   p_hh = ch ph;  en = -(ch ph - p_hh) - ch pl - cl ph  (exact first step)
//   t = h + p_hh, Knuth two-sum error into l together with -en
__device__ __forceinline__ void df_acc2(float2 &h, float2 &l, float2 ch, float2 nch, float2 ncl, float2 ph, float2 pl) {
    const float2 p = __fmul2_rn(ch, ph);
    float2 en = __ffma2_rn(nch, ph, p);
    en = __ffma2_rn(nch, pl, en);
    en = __ffma2_rn(ncl, ph, en);
    const float2 t = __fadd2_rn(h, p);
    const float2 bb = fsub2(t, h);
    const float2 s = __fadd2_rn(fsub2(h, fsub2(t, bb)), fsub2(p, bb));
    l = __fadd2_rn(l, fsub2(s, en));
    h = t;
}
__device__ __forceinline__ void df_add_to2(float2 &h, float2 &l, float2 ph, float2 pl) {
    const float2 t = __fadd2_rn(h, ph);
    const float2 bb = fsub2(t, h);
    l = __fadd2_rn(l, __fadd2_rn(__fadd2_rn(fsub2(h, fsub2(t, bb)), fsub2(ph, bb)), pl));
    h = t;
}

// coefficient pairs of one bond for one thread: hi, -hi, -lo of the
// coefficient at register parity 0 (s) and 1 (f)
struct DfCoef {
    float2 sh, snh, snl, fh, fnh, fnl;
};
template <int LE, int KA, int KB>
__device__ __forceinline__ void bond_apply_df(float2 (&ah)[1 << LE], float2 (&al)[1 << LE], const float2 (&ph)[1 << LE],
                                              const float2 (&pl)[1 << LE], const DfCoef &c) {
    constexpr int E = 1 << LE;
#pragma unroll
    for (int k = 0; k < E; ++k) {
        const int kpar = (KA >= 0 ? (k >> KA) & 1 : 0) ^ (KB >= 0 ? (k >> KB) & 1 : 0);
        const int kp = k ^ KMask<KA, KB>::m;
        if (kpar) df_acc2(ah[k], al[k], c.fh, c.fnh, c.fnl, ph[kp], pl[kp]);
        else df_acc2(ah[k], al[k], c.sh, c.snh, c.snl, ph[kp], pl[kp]);
    }
}

#define FTK_HV_DF_CASE(ID, KA, KB)                                                                   \
    case ID:                                                                                         \
        if constexpr (KA < LE && KB < LE) bond_apply_df<LE, KA, KB>(ah, al, ph, pl, cf);             \
        break;

// TB > 0: the thread bits of the tile (tile_bits - LE) as a compile-time
// constant, so that the strides T k of the shared tile fold into immediate
// offsets (the 2^12-amplitude tiles of the 24-site plans: TB = 9).
template <int LE, int EPI, bool FU, int TB>
__global__ void __launch_bounds__(512, 1)
hv_pass_df_kernel(const float2 *__restrict__ in, float2 *out, const PassDesc pd, const EpiArgs ea) {
    constexpr int E = 1 << LE;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (ea.all_done && *ea.all_done) return;
    if (ea.lowp && *ea.lowp != ea.lowp_run) return;
    if (ea.fu_seed && ea.fu_seed->done != 0) return;   // finished column (COCG): no work
    const long long lo = ea.df_lo;
    const int b = TB > 0 ? TB + LE : pd.tile_bits;
    const int tb = b - LE;
    const int tile_n = 1 << b;
    const int T = 1 << tb;
    const int t = threadIdx.x;
    const bool act = t < T;
    // tile buffers of (hi.re, hi.im, lo.re, lo.im): one 16-byte shared load
    // per partner amplitude
    float4 *b0 = reinterpret_cast<float4 *>(smem_raw);
    float4 *b1 = b0 + tile_n, *pb = b1 + tile_n;
    double *red = reinterpret_cast<double *>(pb + tile_n);

    uint64_t st = 0;
    for (int q = 0; q < tb; ++q)
        if ((t >> q) & 1) st |= 1ull << pd.tile_pos[q];
    long long kofs[LE > 0 ? LE : 1];
#pragma unroll
    for (int q = 0; q < LE; ++q) kofs[q] = (long long)(1ull << pd.tile_pos[tb + q]);
    auto eofs = [&](int k) -> long long {
        long long v = (long long)st;
#pragma unroll
        for (int q = 0; q < LE; ++q)
            if ((k >> q) & 1) v += kofs[q];
        return v;
    };
    // tile offsets: the bits of the tile index deposited at the free sites.
    // Successive tiles of a CTA are gridDim.x apart; their offsets follow by
    // a masked addition (the bits outside the mask set to 1 carry across
    // them): dep(a + g) = ((dep(a) | ~mask) + dep(g)) & mask.
    auto tile_ofs = [&](long tau) -> long long {
        uint64_t v = 0;
        for (int q = 0; q < pd.n_free; ++q)
            if ((tau >> q) & 1) v |= 1ull << pd.free_pos[q];
        return (long long)v;
    };
    // (mask and step in shared memory: read once per tile, no registers held)
    __shared__ uint64_t free_mask, dep_grid;
    if (threadIdx.x == 0) {
        uint64_t m = 0;
        for (int q = 0; q < pd.n_free; ++q) m |= 1ull << pd.free_pos[q];
        free_mask = m;
        dep_grid = (uint64_t)tile_ofs(gridDim.x);
    }
    __syncthreads();
    auto next_ofs = [&](long long ofs) -> long long {
        const uint64_t m = free_mask;
        return (long long)((((uint64_t)ofs | ~m) + dep_grid) & m);
    };
    // diagonal dgv[0] c0 + dgv[1] c1 (integer counts c as in the kernel
    // above) in double-float arithmetic, once per thread
    float dgh[E], dgl[E];
    {
        int c0[E], c1[E];
#pragma unroll
        for (int k = 0; k < E; ++k) { c0[k] = 0; c1[k] = 0; }
        for (int l = 0; l < pd.n_bonds; ++l) {
            const int m = (1 << pd.bi[l]) | (1 << pd.bj[l]);
            const int pt = __popc(t & m & (T - 1)) & 1;
            const int km = m >> tb;
            const int cls = pd.dgc[l];
#pragma unroll
            for (int k = 0; k < E; ++k) {
                const int sg = 1 - 2 * ((pt ^ __popc(k & km)) & 1);
                c0[k] += cls ? 0 : sg;
                c1[k] += cls ? sg : 0;
            }
        }
#pragma unroll
        for (int k = 0; k < E; ++k) {
            const dfl d = dfl_add(dfl_mul({(float)c0[k], 0.f}, {pd.dgv_f[0], pd.dgv_lo[0]}),
                                  dfl_mul({(float)c1[k], 0.f}, {pd.dgv_f[1], pd.dgv_lo[1]}));
            dgh[k] = d.hi;
            dgl[k] = d.lo;
        }
    }
    Acc<float> dot[2];
    const bool first = pd.first != 0;
    // fused residual update (first pass only; a finished column returned above)
    DfUpdDots udots;
    auto issue = [&](const float2 *src, long long tofs, float4 *b) {
        if (act) {
            const float2 *g = src + tofs, *gl = g + lo;
#pragma unroll
            for (int k = 0; k < E; ++k) {
                const long long e = eofs(k);
                float2 *d = reinterpret_cast<float2 *>(b + t + T * k);
                cp_async_elem(d, g + e);
                cp_async_elem(d + 1, gl + e);
            }
        }
        cp_async_commit();
    };
    const long n_tiles = 1L << pd.n_free;
    long tau = blockIdx.x;
    long long tofs = tau < n_tiles ? tile_ofs(tau) : 0;
    if (tau < n_tiles) {
        if (!FU) issue(in, tofs, b0);
        if (!first) issue(out, tofs, pb);
    }
    for (int it = 0; tau < n_tiles; tau += gridDim.x, ++it) {
        const float4 *cb = (it & 1) ? b1 : b0;
        float4 *nb = (it & 1) ? b0 : b1;
        const long tn = tau + gridDim.x;
        const bool more = tn < n_tiles;
        const long long tofs_n = more ? next_ofs(tofs) : 0;
        if (!FU && more) issue(in, tofs_n, nb);
        if (first) { if (more) cp_async_wait<1>(); else cp_async_wait<0>(); }
        else { if (more) cp_async_wait<2>(); else cp_async_wait<1>(); }
        __syncthreads();
        if constexpr (FU) {
            // the tile of r_{k+1}: computed from r_k, r_{k-1}, w_k (all at the
            // tile's own offsets, read before this thread overwrites them),
            // written to r_{k+1}'s buffer and to the current shared buffers
            if (act) {
                float4 *sb = const_cast<float4 *>(cb);
                float2 *rn = ea.fu_rnew + tofs, *rc = ea.fu_rcur + tofs, *wk = out + tofs;
                const float4 *lm = ea.fu_lam + tofs;
                {
                    const DfStep qs = df_step(*ea.fu_seed);
                    // loads of KB elements first (independent, in flight
                    // together), then their arithmetic and stores
                    constexpr int KB = E < 2 ? E : 2;
#pragma unroll
                    for (int k0 = 0; k0 < E; k0 += KB) {
                        float2 ah[KB], al[KB], ph2[KB], pl2[KB], wh[KB], wl[KB];
                        float4 l4[KB];
#pragma unroll
                        for (int u = 0; u < KB; ++u) {
                            const long long e = eofs(k0 + u);
                            ah[u] = rc[e]; al[u] = rc[e + lo]; ph2[u] = rn[e]; pl2[u] = rn[e + lo];
                            wh[u] = wk[e]; wl[u] = wk[e + lo]; l4[u] = lm[e];
                        }
#pragma unroll
                        for (int u = 0; u < KB; ++u) {
                            const int k = k0 + u;
                            const long long e = eofs(k);
                            const dcl r = df_next_residual({{ah[u].x, al[u].x}, {ah[u].y, al[u].y}},
                                                           {{ph2[u].x, pl2[u].x}, {ph2[u].y, pl2[u].y}},
                                                           {{wh[u].x, wl[u].x}, {wh[u].y, wl[u].y}}, qs);
                            if (qs.f != 1.f) {
                                rc[e] = make_float2(ah[u].x * qs.f, ah[u].y * qs.f);
                                rc[e + lo] = make_float2(al[u].x * qs.f, al[u].y * qs.f);
                            }
                            const float2 nh2 = make_float2(r.re.hi, r.im.hi), nl2 = make_float2(r.re.lo, r.im.lo);
                            rn[e] = nh2;
                            rn[e + lo] = nl2;
                            sb[t + T * k] = make_float4(nh2.x, nh2.y, nl2.x, nl2.y);
                            udots.add(r, l4[u]);
                        }
                    }
                }
            }
            __syncthreads();
            // the next tile's update inputs to L2 while this tile's bonds run
            // (one prefetch per 128-byte line: every 16th lane for float2
            // arrays, every 8th for the float4 lambda)
            if (act && more) {
                const int lane = t & 31;
#pragma unroll
                for (int k = 0; k < E; ++k) {
                    const long long e = tofs_n + eofs(k);
                    if ((lane & 15) == 0) {
                        prefetch_l2(ea.fu_rcur + e); prefetch_l2(ea.fu_rcur + e + lo);
                        prefetch_l2(ea.fu_rnew + e); prefetch_l2(ea.fu_rnew + e + lo);
                        prefetch_l2(out + e); prefetch_l2(out + e + lo);
                    }
                    if ((lane & 7) == 0) prefetch_l2(ea.fu_lam + e);
                }
            }
        }
        if (act) {
            float2 ah[E], al[E];   // (re, im) hi and lo parts of the accumulators
            float2 ph[E], pl[E];
#pragma unroll
            for (int k = 0; k < E; ++k) { ah[k] = make_float2(0.f, 0.f); al[k] = make_float2(0.f, 0.f); }
            int q = 0;
            for (int g = 0; g < pd.n_groups; ++g) {
                const int tm = pd.grp_tmask[g];
#pragma unroll
                for (int k = 0; k < E; ++k) {
                    const float4 v4 = cb[(t ^ tm) + T * k];
                    ph[k] = make_float2(v4.x, v4.y);
                    pl[k] = make_float2(v4.z, v4.w);
                }
                const int pt = __popc(t & tm) & 1;
                for (const int end = pd.grp_end[g]; q < end; ++q) {
                    const float parh = pd.par_f[q], parl = pd.par_lo[q], anth = pd.anti_f[q], antl = pd.anti_lo[q];
                    const float sh_ = pt ? anth : parh, sl_ = pt ? antl : parl;
                    const float fh_ = pt ? parh : anth, fl_ = pt ? parl : antl;
                    const DfCoef cf = {make_float2(sh_, sh_), make_float2(-sh_, -sh_), make_float2(-sl_, -sl_),
                                       make_float2(fh_, fh_), make_float2(-fh_, -fh_), make_float2(-fl_, -fl_)};
                    switch (pd.bcase[q]) {
                        FTK_HV_DF_CASE(0, -1, -1)
                        FTK_HV_DF_CASE(1, 0, -1)
                        FTK_HV_DF_CASE(2, 1, -1)
                        FTK_HV_DF_CASE(3, 2, -1)
                        FTK_HV_DF_CASE(4, 3, -1)
                        FTK_HV_DF_CASE(9 + 0 * 8 + 1, 0, 1)
                        FTK_HV_DF_CASE(9 + 0 * 8 + 2, 0, 2)
                        FTK_HV_DF_CASE(9 + 0 * 8 + 3, 0, 3)
                        FTK_HV_DF_CASE(9 + 1 * 8 + 2, 1, 2)
                        FTK_HV_DF_CASE(9 + 1 * 8 + 3, 1, 3)
                        FTK_HV_DF_CASE(9 + 2 * 8 + 3, 2, 3)
                        default: break;
                    }
                }
            }
            // own amplitudes (last group): diagonal
#pragma unroll
            for (int k = 0; k < E; ++k)
                df_acc2(ah[k], al[k], make_float2(dgh[k], dgh[k]), make_float2(-dgh[k], -dgh[k]),
                        make_float2(-dgl[k], -dgl[k]), ph[k], pl[k]);
            if (!first) {
                if (more) cp_async_wait<1>(); else cp_async_wait<0>();
#pragma unroll
                for (int k = 0; k < E; ++k) {
                    const float4 v4 = pb[t + T * k];
                    df_add_to2(ah[k], al[k], make_float2(v4.x, v4.y), make_float2(v4.z, v4.w));
                }
            }
            float2 *o = out + tofs, *ol = o + lo;
#pragma unroll
            for (int k = 0; k < E; ++k) {
                // renormalise (fast two-sum) and store hi, lo
                const float2 hh = __fadd2_rn(ah[k], al[k]);
                const float2 ll = fsub2(al[k], fsub2(hh, ah[k]));
                const long long e = eofs(k);
                o[e] = hh;
                ol[e] = ll;
                if (EPI == EPI_COCG && pd.last) {
                    // mu = r^T w (bilinear) in double-float from hi + lo
                    dot[0].fma_pair(ph[k].x, pl[k].x, hh.x, ll.x);
                    dot[0].fma_pair(-ph[k].y, -pl[k].y, hh.y, ll.y);
                    dot[1].fma_pair(ph[k].x, pl[k].x, hh.y, ll.y);
                    dot[1].fma_pair(ph[k].y, pl[k].y, hh.x, ll.x);
                }
            }
        }
        if (!first && more) issue(out, tofs_n, pb);
        tofs = tofs_n;
        __syncthreads();
    }
    cp_async_wait<0>();
    if constexpr (FU) {
        // update dots of r_{k+1} (and mu when this pass is also the last)
        double v[7];
        udots.get(*reinterpret_cast<double(*)[5]>(v));
        v[5] = (EPI == EPI_COCG) ? dot[0].get() : 0.0;
        v[6] = (EPI == EPI_COCG) ? dot[1].get() : 0.0;
        block_reduce<7>(v, red);
        if (threadIdx.x < 7) ea.partials[(size_t)blockIdx.x * 7 + threadIdx.x] = red[threadIdx.x];
        __shared__ double fin[7];
        if (!last_block_reduce<7>(ea.partials, ea.counter, fin, red)) return;
        if (threadIdx.x < 5) ea.fu_result[threadIdx.x] = fin[threadIdx.x];
        if (EPI == EPI_COCG && pd.last && threadIdx.x < 2) ea.result[threadIdx.x] = fin[5 + threadIdx.x];
        return;
    }
    if (EPI != EPI_COCG || !pd.last) return;
    double v[2] = {dot[0].get(), dot[1].get()};
    block_reduce<2>(v, red);
    if (threadIdx.x < 2) ea.partials[(size_t)blockIdx.x * 2 + threadIdx.x] = red[threadIdx.x];
    last_block_reduce<2>(ea.partials, ea.counter, ea.result, red);
}

// ===================================================================== host
// Register bits per thread: 16 (FP32) or 8 (FP64) amplitude-RHS pairs of
// accumulators, i.e. le = log2(16 / B) or log2(8 / B), with at most 512
// threads per CTA (128 registers). Right-hand-side blocks wider than 8 run
// in column chunks of 8. (32 pairs with 256 threads measured no faster.)
static int log2i(int v) {
    int r = 0;
    while ((1 << (r + 1)) <= v) ++r;
    return r;
}
int hv_max_b(int prec) { return prec == 2 ? 1 : 8; }
static int hv_le_default(int prec, int B) {
    const int bc = std::min(B, hv_max_b(prec));
    return std::max(0, (prec == 1 ? 4 : 3) - log2i(bc));
}
int hv_le(int prec, int B, int tile_bits, int chunk_bits) {
    const int le = hv_le_default(prec, B);
    if (tile_bits - le < 5 || tile_bits - le < chunk_bits) return 0;
    return le;
}
// Largest tile: 64 KB (three such buffers per CTA: two for the input, one
// for the partial product) and at most 512 threads.
int hv_max_tile_bits(int prec, int B) {
    const int bc = std::min(B, hv_max_b(prec));
    const int es = prec == 1 ? 8 : 16;   // FP64 and double-float: 16 B per amplitude
    int tb = 0;
    while ((size_t(2) << tb) * bc * es <= (size_t(64) << 10)) ++tb;
    return std::min(tb, 9 + hv_le_default(prec, B));
}
int hv_threads(const PassDesc &pd) {
    const int t = 1 << (pd.tile_bits - pd.le);
    return t < 32 ? 32 : t;
}
size_t hv_smem_bytes(int prec, int B, const PassDesc &pd) {
    const int bc = std::min(B, hv_max_b(prec));
    const size_t es = prec == 1 ? 8 : 16;
    const int nd = prec == 2 ? 8 : std::max(2, 2 * bc);   // double-float: fused update dots + mu
    return size_t(3) * ((size_t)1 << pd.tile_bits) * bc * es + (size_t)(hv_threads(pd) / 32) * nd * 8;
}

// Choose the register sites of a planned pass and order its bonds in groups.
// The register sites are le of the non-chunk tile sites, picked to minimise
// the number of groups (shared-memory reads per amplitude); the offset bits
// are renumbered chunk sites, other thread sites, register sites.
bool hv_layout_pass(PassDesc &pd, int prec, int B) {
    const int b = pd.tile_bits, c = pd.chunk_bits, nb = pd.n_bonds;
    if (B < 1 || B > hv_max_b(prec) || (B & (B - 1))) return false;
    const int le = hv_le(prec, B, b, c);
    const int tb = b - le;
    // choose the register positions among offset bits [c, b)
    const int free_n = b - c;
    int best_set = -1, best_groups = 1 << 30, best_rr = -1;
    for (int set = 0; set < (1 << free_n); ++set) {
        if (__builtin_popcount(set) != le) continue;
        // bond masks with the chosen offset bits counted as register bits
        int tms[FTK_MAX_PASS_BONDS + 1];
        int ng = 0, rr = 0;
        for (int l = 0; l < nb; ++l) {
            int tm = 0, nreg = 0;
            for (int side = 0; side < 2; ++side) {
                const int o = side ? pd.bj[l] : pd.bi[l];
                const bool reg = o >= c && ((set >> (o - c)) & 1);
                if (reg) ++nreg;
                else tm |= 1 << o;   // thread masks compared as sets of offset bits
            }
            if (nreg == 2) ++rr;
            bool seen = tm == 0;
            for (int g = 0; g < ng && !seen; ++g) seen = tms[g] == tm;
            if (!seen) tms[ng++] = tm;
        }
        ++ng;   // the own group
        if (ng < best_groups || (ng == best_groups && rr > best_rr)) {
            best_groups = ng;
            best_rr = rr;
            best_set = set;
        }
        if (free_n > 20) break;
    }
    if (best_set < 0) return false;
    // renumber offset bits: chunk bits, other thread bits, register bits
    int newpos[FTK_MAX_TILE_BITS];
    int nt = 0;
    for (int o = 0; o < c; ++o) newpos[o] = nt++;
    for (int o = c; o < b; ++o)
        if (!((best_set >> (o - c)) & 1)) newpos[o] = nt++;
    for (int o = c; o < b; ++o)
        if ((best_set >> (o - c)) & 1) newpos[o] = nt++;
    if (nt != b || (b - le) != tb) return false;
    PassDesc q = pd;
    for (int o = 0; o < b; ++o) q.tile_pos[newpos[o]] = pd.tile_pos[o];
    // bonds with their new offset bits, grouped by thread mask (own group last)
    int tmask[FTK_MAX_PASS_BONDS];
    for (int l = 0; l < nb; ++l) {
        const int bi = newpos[pd.bi[l]], bj = newpos[pd.bj[l]];
        tmask[l] = ((1 << bi) | (1 << bj)) & ((1 << tb) - 1);
    }
    // stable order: distinct nonzero masks in first-appearance order, then 0
    int gm[FTK_MAX_PASS_BONDS + 1], ng = 0;
    for (int l = 0; l < nb; ++l) {
        if (tmask[l] == 0) continue;
        bool seen = false;
        for (int g = 0; g < ng; ++g) seen |= gm[g] == tmask[l];
        if (!seen) gm[ng++] = tmask[l];
    }
    gm[ng++] = 0;
    int w = 0;
    for (int g = 0; g < ng; ++g) {
        for (int l = 0; l < nb; ++l) {
            if (tmask[l] != gm[g]) continue;
            const int bi = newpos[pd.bi[l]], bj = newpos[pd.bj[l]];
            q.bi[w] = bi;
            q.bj[w] = bj;
            q.par[w] = pd.par[l];
            q.anti[w] = pd.anti[l];
            q.par_f[w] = pd.par_f[l];
            q.anti_f[w] = pd.anti_f[l];
            q.par_lo[w] = pd.par_lo[l];
            q.anti_lo[w] = pd.anti_lo[l];
            q.dgc[w] = pd.dgc[l];
            const int km = ((1 << bi) | (1 << bj)) >> tb;
            int ka = -1, kb = -1;
            for (int a = 0; a < le; ++a)
                if ((km >> a) & 1) { if (ka < 0) ka = a; else kb = a; }
            q.bcase[w] = (int8_t)(ka < 0 ? 0 : kb < 0 ? 1 + ka : 9 + 8 * ka + kb);
            ++w;
        }
        q.grp_tmask[g] = gm[g];
        q.grp_end[g] = w;
    }
    if (w != nb) return false;
    q.n_groups = ng;
    q.le = le;
    q.cols = B;
    pd = q;
    return true;
}

template <typename K>
static cudaError_t opt_in(K kern) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    return e;
}

template <typename R, int B, int LE, int TB>
static cudaError_t attrs_le_tb() {
    cudaError_t e = opt_in(hv_pass_kernel<R, B, LE, EPI_PLAIN, TB>);
    if (e == cudaSuccess) e = opt_in(hv_pass_kernel<R, B, LE, EPI_COCG, TB>);
    if constexpr (sizeof(R) == 4)
        if (e == cudaSuccess) e = opt_in(hv_pass_kernel<R, B, LE, EPI_COCG_MIXED, TB>);
    if constexpr (B == 1)
        if (e == cudaSuccess) e = opt_in(hv_pass_kernel<R, 1, LE, EPI_TPQ, TB>);
    if constexpr (B == 1 && sizeof(R) == 8)
        if (e == cudaSuccess) e = opt_in(hv_pass_kernel<R, 1, LE, EPI_TAYLOR, TB>);
    return e;
}
template <typename R, int B, int LE>
static cudaError_t attrs_le() {
    cudaError_t e = attrs_le_tb<R, B, LE, 0>();
    if constexpr (B == 1 && LE > 0)
        if (e == cudaSuccess) e = attrs_le_tb<R, 1, LE, 9>();
    return e;
}

template <typename R, int B, int LEDEF>
static cudaError_t attrs_b() {
    cudaError_t e = attrs_le<R, B, LEDEF>();
    if (e == cudaSuccess && LEDEF != 0) e = attrs_le<R, B, 0>();
    return e;
}

// Opt every H.V pass instantiation into the full shared memory once per
// process (outside any stream capture); thread-safe (contexts may be created
// from several host threads, as the server does).
template <int LE, int TB>
static cudaError_t attrs_df() {
    cudaError_t e = opt_in(hv_pass_df_kernel<LE, EPI_PLAIN, false, TB>);
    if (e == cudaSuccess) e = opt_in(hv_pass_df_kernel<LE, EPI_COCG, false, TB>);
    if (e == cudaSuccess) e = opt_in(hv_pass_df_kernel<LE, EPI_PLAIN, true, TB>);
    if (e == cudaSuccess) e = opt_in(hv_pass_df_kernel<LE, EPI_COCG, true, TB>);
    return e;
}

static cudaError_t init_attributes_once() {
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = attrs_df<3, 0>();
    if (e == cudaSuccess) e = attrs_df<3, 9>();
    if (e == cudaSuccess) e = attrs_df<0, 0>();
    if (e == cudaSuccess) e = attrs_b<double, 1, 3>();
    if (e == cudaSuccess) e = attrs_b<double, 2, 2>();
    if (e == cudaSuccess) e = attrs_b<double, 4, 1>();
    if (e == cudaSuccess) e = attrs_b<double, 8, 0>();
    if (e == cudaSuccess) e = attrs_b<float, 1, 4>();
    if (e == cudaSuccess) e = attrs_b<float, 2, 3>();
    if (e == cudaSuccess) e = attrs_b<float, 4, 2>();
    if (e == cudaSuccess) e = attrs_b<float, 8, 1>();
    return e;
}

cudaError_t init_kernel_attributes() {
    static std::once_flag once;
    static cudaError_t status = cudaSuccess;
    std::call_once(once, [] { status = init_attributes_once(); });
    return status;
}

template <typename R, int B, int LE, int TB>
static void (*pass_kernel(int epi))(const typename C2<R>::t *, typename C2<R>::t *, long long, const PassDesc,
                                    const EpiArgs) {
    if (epi == EPI_PLAIN) return hv_pass_kernel<R, B, LE, EPI_PLAIN, TB>;
    if (epi == EPI_COCG) return hv_pass_kernel<R, B, LE, EPI_COCG, TB>;
    if constexpr (sizeof(R) == 4)
        if (epi == EPI_COCG_MIXED) return hv_pass_kernel<R, B, LE, EPI_COCG_MIXED, TB>;
    if constexpr (B == 1) {
        if (epi == EPI_TPQ) return hv_pass_kernel<R, 1, LE, EPI_TPQ, TB>;
        if constexpr (sizeof(R) == 8)
            if (epi == EPI_TAYLOR) return hv_pass_kernel<R, 1, LE, EPI_TAYLOR, TB>;
    }
    return nullptr;
}

template <typename R, int B, int LE>
static cudaError_t launch_le(int epi, const void *in, void *out, long long ld, const PassDesc &pd, const EpiArgs &ea,
                             int grid_cap, cudaStream_t st) {
    typedef typename C2<R>::t cx;
    void (*k)(const cx *, cx *, long long, const PassDesc, const EpiArgs) = pass_kernel<R, B, LE, 0>(epi);
    if constexpr (B == 1 && LE > 0)
        if (pd.tile_bits == 9 + LE) k = pass_kernel<R, 1, LE, 9>(epi);
    if (!k) return cudaErrorInvalidValue;
    const int threads = hv_threads(pd);
    const size_t smem = hv_smem_bytes(sizeof(R) == 8 ? 0 : 1, pd.cols, pd);
    // persistent grid: the CTAs that are resident at once
    int per_sm = 0, dev = 0, n_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long n_tiles = 1L << pd.n_free;
    long g = (long)per_sm * n_sm;
    if (g > n_tiles) g = n_tiles;
    if (g > grid_cap) g = grid_cap;   // the caller's partial buffers
    k<<<(int)g, threads, smem, st>>>(reinterpret_cast<const cx *>(in), reinterpret_cast<cx *>(out), ld, pd, ea);
    return cudaGetLastError();
}

template <typename R, int B, int LEDEF>
static cudaError_t launch_b(int epi, const void *in, void *out, long long ld, const PassDesc &pd, const EpiArgs &ea,
                            int grid_cap, cudaStream_t st) {
    if (pd.le == LEDEF) return launch_le<R, B, LEDEF>(epi, in, out, ld, pd, ea, grid_cap, st);
    if (pd.le == 0) return launch_le<R, B, 0>(epi, in, out, ld, pd, ea, grid_cap, st);
    return cudaErrorInvalidValue;
}

template <typename R>
static cudaError_t launch_chunk(int bc, int epi, const void *in, void *out, long long ld, const PassDesc &pd,
                                const EpiArgs &ea, int grid_cap, cudaStream_t st) {
    if constexpr (sizeof(R) == 4) {
        switch (bc) {
        case 1: return launch_b<R, 1, 4>(epi, in, out, ld, pd, ea, grid_cap, st);
        case 2: return launch_b<R, 2, 3>(epi, in, out, ld, pd, ea, grid_cap, st);
        case 4: return launch_b<R, 4, 2>(epi, in, out, ld, pd, ea, grid_cap, st);
        case 8: return launch_b<R, 8, 1>(epi, in, out, ld, pd, ea, grid_cap, st);
        default: return cudaErrorInvalidValue;
        }
    } else {
        switch (bc) {
        case 1: return launch_b<R, 1, 3>(epi, in, out, ld, pd, ea, grid_cap, st);
        case 2: return launch_b<R, 2, 2>(epi, in, out, ld, pd, ea, grid_cap, st);
        case 4: return launch_b<R, 4, 1>(epi, in, out, ld, pd, ea, grid_cap, st);
        case 8: return launch_b<R, 8, 0>(epi, in, out, ld, pd, ea, grid_cap, st);
        default: return cudaErrorInvalidValue;
        }
    }
}

template <int LE, int TB>
static void (*df_kernel(int epi, bool fu))(const float2 *, float2 *, const PassDesc, const EpiArgs) {
    return epi == EPI_COCG
               ? (fu ? hv_pass_df_kernel<LE, EPI_COCG, true, TB> : hv_pass_df_kernel<LE, EPI_COCG, false, TB>)
               : (fu ? hv_pass_df_kernel<LE, EPI_PLAIN, true, TB> : hv_pass_df_kernel<LE, EPI_PLAIN, false, TB>);
}

template <int LE>
static cudaError_t launch_df_le(int epi, const void *in, void *out, const PassDesc &pd, const EpiArgs &ea,
                                int grid_cap, cudaStream_t st) {
    const bool fu = ea.fu_seed != nullptr && pd.first;
    void (*k)(const float2 *, float2 *, const PassDesc, const EpiArgs) = df_kernel<LE, 0>(epi, fu);
    if constexpr (LE == 3)
        if (pd.tile_bits == 12) k = df_kernel<LE, 9>(epi, fu);
    const int threads = hv_threads(pd);
    const size_t smem = hv_smem_bytes(2, 1, pd);
    int per_sm = 0, dev = 0, n_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long g = std::min<long>((long)per_sm * n_sm, 1L << pd.n_free);
    if (g > grid_cap) g = grid_cap;
    k<<<(int)g, threads, smem, st>>>(reinterpret_cast<const float2 *>(in), reinterpret_cast<float2 *>(out), pd, ea);
    return cudaGetLastError();
}

// Double-float passes: B columns, one launch each; column j's hi array at
// j 2^N, its lo array ea.df_lo float2 later (both for in and out).
static cudaError_t launch_hv_pass_df(int B, int epi, const void *in, void *out, const PassDesc &pd,
                                     const EpiArgs &ea, int grid_cap, cudaStream_t st) {
    if (epi != EPI_PLAIN && epi != EPI_COCG) return cudaErrorInvalidValue;
    const long long ld = 1LL << pd.n_sites;
    for (int j = 0; j < B; ++j) {
        EpiArgs e = ea;
        if (e.result) e.result += 2 * j;
        if (e.fu_seed) {   // fused residual update: this column's vectors, seed and dots
            e.fu_seed += j;
            e.fu_rcur += (size_t)j * ld;
            e.fu_rnew = static_cast<float2 *>(const_cast<void *>(in)) + (size_t)j * ld;
            e.fu_lam += (size_t)j * ld;
            e.fu_result += (size_t)FTK_UPD_DOTS * j;
        }
        const void *i = static_cast<const float2 *>(in) + (size_t)j * ld;
        void *o = static_cast<float2 *>(out) + (size_t)j * ld;
        const cudaError_t r = pd.le == 3 ? launch_df_le<3>(epi, i, o, pd, e, grid_cap, st)
                                         : launch_df_le<0>(epi, i, o, pd, e, grid_cap, st);
        if (r != cudaSuccess) return r;
    }
    return cudaSuccess;
}

cudaError_t launch_hv_pass(int prec, int B, int epi, const void *in, void *out, const PassDesc &pd,
                           const EpiArgs &ea, int grid_cap, cudaStream_t st) {
    const int bc = pd.cols;
    if (B < 1 || (B & (B - 1)) || B > FTK_MAX_RHS || bc < 1 || bc > hv_max_b(prec) || (B % bc) ||
        pd.le != hv_le(prec, bc, pd.tile_bits, pd.chunk_bits) || hv_threads(pd) > 512 ||
        ((epi == EPI_TPQ || epi == EPI_TAYLOR) && B != 1) || (epi == EPI_TAYLOR && (prec != 0 || !ea.taylor_acc)) ||
        (ea.lo && prec != 1) || (prec == 2 && ea.df_lo <= 0))
        return cudaErrorInvalidConfiguration;
    if (prec == 2) return launch_hv_pass_df(B, epi, in, out, pd, ea, grid_cap, st);
    const size_t es = prec == 0 ? 16 : 8;
    for (int j0 = 0; j0 < B; j0 += bc) {
        EpiArgs e = ea;
        if (e.result) e.result += 2 * j0;   // COCG: mu of columns j0 .. j0 + bc
        if (e.lo) e.lo = static_cast<const char *>(e.lo) + (size_t)j0 * (1LL << pd.n_sites) * es;
        const long long ld = 1LL << pd.n_sites;   // column stride: one vector
        const void *i = static_cast<const char *>(in) + (size_t)j0 * ld * es;
        void *o = static_cast<char *>(out) + (size_t)j0 * ld * es;
        const int ep = (epi == EPI_COCG && e.lo && pd.last) ? EPI_COCG_MIXED : epi;
        const cudaError_t r = prec == 0 ? launch_chunk<double>(bc, ep, i, o, ld, pd, e, grid_cap, st)
                                        : launch_chunk<float>(bc, ep, i, o, ld, pd, e, grid_cap, st);
        if (r != cudaSuccess) return r;
    }
    return cudaSuccess;
}

}  // namespace ftk
