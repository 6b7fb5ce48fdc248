// CUDA kernels of the FTKomega hot path (sm_103a). No tensor cores: the
// Hamiltonian-vector product is a bit-indexed gather, not a contraction.
//
//   hv_pass     one tiled pass of H.V (Sec. IV.A "Lanczos step"), fused
//               epilogues for the mTPQ step (Appendix A) and the COCG mu dot
//   cocg_update 3-term seed-COCG residual update with fused dots (Sec. II.B)
//   cocg_seed   per-RHS seed scalars alpha_k, c_k and convergence test
//   cocg_shift  per-shift recurrences pi, alpha^s, beta^s, projected p, G
//   apply_op    S^gamma_q probe (Sec. V)
//   init_state  Philox4x32-10 + Box-Muller random state (Sec. II.A)
//   spectrum    reweighting of shells to temperatures (Eq. B1 reading R1)
//
// All reductions are deterministic: per-CTA partials in a fixed order, then
// the last CTA to finish (ticket from an integer atomic) sums the partials in
// a fixed order and writes the result. No floating-point atomics.
#include "ftk_common.cuh"
#include "ftk_kernels.h"

#include <math.h>

namespace ftk {

// ---------------------------------------------------------------- complex
template <typename R> struct C2;
template <> struct C2<double> { typedef double2 t; };
template <> struct C2<float> { typedef float2 t; };

template <typename R>
__device__ __forceinline__ typename C2<R>::t mk(R a, R b) {
    typename C2<R>::t z; z.x = a; z.y = b; return z;
}

// ------------------------------------------------ per-thread dot accumulator
// double: plain sum. float: the product of two floats is split exactly into
// p + e with an FMA (two-product) and both parts enter a Knuth two-sum
// compensated float accumulator, converted to double once per thread.
template <typename R> struct Acc;
template <> struct Acc<double> {
    double s;
    __device__ Acc() : s(0.0) {}
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ void fma2(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double get() const { return s; }
};
template <> struct Acc<float> {
    float s, c;
    __device__ Acc() : s(0.f), c(0.f) {}
    __device__ __forceinline__ void add(float v) {
        float t = s + v;
        float bp = t - s;
        float err = (s - (t - bp)) + (v - bp);
        s = t;
        c += err;
    }
    __device__ __forceinline__ void fma2(float a, float b) {
        float p = a * b;
        float e = fmaf(a, b, -p);
        add(p);
        c += e;
    }
    __device__ __forceinline__ double get() const { return (double)s + (double)c; }
};

// ---------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Reduce nd values per thread over the block (fixed order) into red[0..nd).
// red must hold (blockDim/32) * nd doubles. Result valid in red[0..nd) after
// the trailing __syncthreads.
template <int ND>
__device__ void block_reduce(double (&v)[ND], double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int d = 0; d < ND; ++d) v[d] = warp_sum(v[d]);
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int d = 0; d < ND; ++d) red[warp * ND + d] = v[d];
    }
    __syncthreads();
    if (threadIdx.x < ND) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += red[w * ND + threadIdx.x];
        red[threadIdx.x] = s;   // each thread reads column tid, writes slot tid
    }
    __syncthreads();
}

// Called by every thread of every CTA after it stored its ND partials at
// partials[blockIdx.x * ND + d]. Returns true in the (unique) last CTA, after
// it reduced all partials into out[0..ND) in a fixed order. Resets counter.
template <int ND>
__device__ bool last_block_reduce(const double *partials, unsigned int *counter, double *out,
                                  double *red) {
    __shared__ int am_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) am_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!am_last) return false;
    __threadfence();
    double v[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) v[d] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
        for (int d = 0; d < ND; ++d) v[d] += __ldcg(partials + (size_t)b * ND + d);
    }
    block_reduce<ND>(v, red);
    if (threadIdx.x < ND) out[threadIdx.x] = red[threadIdx.x];
    if (threadIdx.x == 0) *counter = 0u;
    __syncthreads();
    return true;
}

// Bond coefficients in the kernel's arithmetic type (no per-element conversion).
template <typename R> struct Coef;
template <> struct Coef<double> {
    __device__ static __forceinline__ double par(const PassDesc &p, int l) { return p.par[l]; }
    __device__ static __forceinline__ double anti(const PassDesc &p, int l) { return p.anti[l]; }
    __device__ static __forceinline__ double dgv(const PassDesc &p, int c) { return p.dgv[c]; }
};
template <> struct Coef<float> {
    __device__ static __forceinline__ float par(const PassDesc &p, int l) { return p.par_f[l]; }
    __device__ static __forceinline__ float anti(const PassDesc &p, int l) { return p.anti_f[l]; }
    __device__ static __forceinline__ float dgv(const PassDesc &p, int c) { return p.dgv_f[c]; }
};

// ------------------------------------------------------------ H.V pass
// Tile offset o (0 <= o < 2^b) -> global index base(t) + (o & chunk) | hi[o >> c].
// Each thread owns offsets o = tid, tid + nthreads, ...; B right-hand sides
// per amplitude are stored contiguously (layout [2^N][B]).
template <typename R, int B, int EPI>
__global__ void __launch_bounds__(B >= 8 ? 256 : 512)
hv_pass_kernel(const typename C2<R>::t *__restrict__ in, typename C2<R>::t *out,
               const PassDesc pd, const EpiArgs ea) {
    typedef typename C2<R>::t cx;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (ea.all_done && *ea.all_done) return;
    const int b = pd.tile_bits, c = pd.chunk_bits;
    const int tile_n = 1 << b;
    const int n_hi = 1 << (b - c);
    cx *tile = reinterpret_cast<cx *>(smem_raw);
    uint32_t *hi = reinterpret_cast<uint32_t *>(smem_raw + (size_t)tile_n * B * sizeof(cx));
    double *red = reinterpret_cast<double *>(hi + n_hi + (n_hi & 1));

    for (int h = threadIdx.x; h < n_hi; h += blockDim.x) {
        uint32_t off = 0;
        for (int k = 0; k < b - c; ++k)
            if ((h >> k) & 1) off |= 1u << pd.tile_pos[c + k];
        hi[h] = off;
    }
    const R scale = (EPI == EPI_TPQ) ? (R)(*ea.scale) : (R)1;
    const R ell = (R)ea.ell, inv_n = (R)ea.inv_n;
    constexpr int ND = (EPI == EPI_TPQ) ? 2 : (EPI == EPI_COCG ? 2 * B : 1);
    Acc<R> dot[ND];

    const long n_tiles = 1L << pd.n_free;
    const uint32_t cmask = (1u << c) - 1u;
    for (long t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        uint64_t base = 0;
        for (int k = 0; k < pd.n_free; ++k)
            if ((t >> k) & 1) base |= 1ull << pd.free_pos[k];
        __syncthreads();   // hi[] ready / previous tile consumed
        for (int idx = threadIdx.x; idx < tile_n * B; idx += blockDim.x) {
            const int o = idx / B, j = idx % B;
            const uint64_t x = base + ((o & cmask) | hi[o >> c]);
            tile[idx] = in[x * B + j];
        }
        __syncthreads();
        for (int o = threadIdx.x; o < tile_n; o += blockDim.x) {
            const uint64_t x = base + ((o & cmask) | hi[o >> c]);
            R ar[B], ai[B];
            if (pd.first) {
#pragma unroll
                for (int j = 0; j < B; ++j) { ar[j] = 0; ai[j] = 0; }
            } else {
#pragma unroll
                for (int j = 0; j < B; ++j) { cx p = out[x * B + j]; ar[j] = p.x; ai[j] = p.y; }
            }
            int c0 = 0, c1 = 0;
            for (int l = 0; l < pd.n_bonds; ++l) {
                const int bi = pd.bi[l], bj = pd.bj[l];
                const int anti = ((o >> bi) ^ (o >> bj)) & 1;
                const R coef = anti ? Coef<R>::anti(pd, l) : Coef<R>::par(pd, l);
                const int sgn = 1 - 2 * anti;
                if (pd.dgc[l]) c1 += sgn; else c0 += sgn;
                const int po = o ^ (1 << bi) ^ (1 << bj);
#pragma unroll
                for (int j = 0; j < B; ++j) {
                    cx p = tile[po * B + j];
                    ar[j] = fma(coef, p.x, ar[j]);
                    ai[j] = fma(coef, p.y, ai[j]);
                }
            }
            const R dsum = Coef<R>::dgv(pd, 0) * (R)c0 + Coef<R>::dgv(pd, 1) * (R)c1;
#pragma unroll
            for (int j = 0; j < B; ++j) {
                cx v = tile[o * B + j];
                ar[j] = fma(dsum, v.x, ar[j]);
                ai[j] = fma(dsum, v.y, ai[j]);
            }
            if (!pd.last || EPI == EPI_PLAIN) {
#pragma unroll
                for (int j = 0; j < B; ++j) out[x * B + j] = mk<R>(ar[j], ai[j]);
            } else if (EPI == EPI_TPQ) {
                // psi' = s (l v - H v / N);  <v|Hv>, |psi'|^2
                cx v = tile[o];
                R yr = scale * (ell * v.x - inv_n * ar[0]);
                R yi = scale * (ell * v.y - inv_n * ai[0]);
                out[x] = mk<R>(yr, yi);
                dot[0].fma2(v.x, ar[0]);
                dot[0].fma2(v.y, ai[0]);
                dot[1].fma2(yr, yr);
                dot[1].fma2(yi, yi);
            } else {
                // W = H R;  mu_j = R_j^T W_j (bilinear)
#pragma unroll
                for (int j = 0; j < B; ++j) {
                    cx v = tile[o * B + j];
                    out[x * B + j] = mk<R>(ar[j], ai[j]);
                    dot[2 * j].fma2(v.x, ar[j]);
                    dot[2 * j].fma2(-v.y, ai[j]);
                    dot[2 * j + 1].fma2(v.x, ai[j]);
                    dot[2 * j + 1].fma2(v.y, ar[j]);
                }
            }
        }
    }
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
        TpqState *st = ea.tpq;
        const double s = st->scale, n = st->n_sites, l = st->ell;
        const double u = s * s * res[0] / n;
        const double q2 = res[1];
        const int k = st->k;
        ea.stat_u[k] = u;
        ea.stat_logq[k] = st->logQ;
        ea.stat_h2[k] = n * n * (q2 - l * l + 2.0 * l * u);
        st->logQ += 0.5 * log(q2);
        st->scale = 1.0 / sqrt(q2);
        st->k = k + 1;
    }
}

// --------------------------------------------------------- COCG update
// mode 0: R_new = lambda_j (start);  mode 1: 3-term seed residual update
//   r_{k+1} = (1 + c_k) r_k - alpha_k (z_s r_k - w_k) - c_k r_{k-1}
// written over r_{k-1}. Fused dots of r_{k+1}: rho = r^T r, g = lambda^dag r,
// |r|^2 (per RHS, FTK_UPD_DOTS doubles each).
template <typename R, int B>
__global__ void __launch_bounds__(256)
cocg_update_kernel(const typename C2<R>::t *__restrict__ rcur, const typename C2<R>::t *__restrict__ w,
                   typename C2<R>::t *rprev_new, UpdArgs ua) {
    typedef typename C2<R>::t cx;
    __shared__ double red[(256 / 32) * FTK_UPD_DOTS * B];
    if (*ua.all_done) return;
    const uint64_t total = ua.dim * B;
    const int j = threadIdx.x % B;     // blockDim and stride are multiples of B
    R a_re = 1, a_im = 0, b_re = 0, b_im = 0, c_re = 0, c_im = 0;
    if (ua.mode == 1) {
        const CocgSeed &s = ua.seed[j];
        // a = 1 + c - alpha z_s, b = alpha, c' = -c
        a_re = (R)(1.0 + s.c_re - (s.alpha_re * s.zs_re - s.alpha_im * s.zs_im));
        a_im = (R)(s.c_im - (s.alpha_re * s.zs_im + s.alpha_im * s.zs_re));
        b_re = (R)s.alpha_re; b_im = (R)s.alpha_im;
        c_re = (R)(-s.c_re); c_im = (R)(-s.c_im);
    }
    const cx *lam = reinterpret_cast<const cx *>(ua.lambda[j]);
    Acc<R> d_rr, d_ri, d_gr, d_gi, d_n;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t x = i / B;
        const cx l = lam[x];
        cx r;
        if (ua.mode == 0) {
            r = l;
        } else {
            const cx rc = rcur[i], wc = w[i], rp = rprev_new[i];
            R re = a_re * rc.x - a_im * rc.y;
            R im = a_re * rc.y + a_im * rc.x;
            re = fma(b_re, wc.x, re); re = fma(-b_im, wc.y, re);
            im = fma(b_re, wc.y, im); im = fma(b_im, wc.x, im);
            re = fma(c_re, rp.x, re); re = fma(-c_im, rp.y, re);
            im = fma(c_re, rp.y, im); im = fma(c_im, rp.x, im);
            r = mk<R>(re, im);
        }
        rprev_new[i] = r;
        d_rr.fma2(r.x, r.x); d_rr.fma2(-r.y, r.y);
        d_ri.fma2(2 * r.x, r.y);
        d_gr.fma2(l.x, r.x); d_gr.fma2(l.y, r.y);
        d_gi.fma2(l.x, r.y); d_gi.fma2(-l.y, r.x);
        d_n.fma2(r.x, r.x); d_n.fma2(r.y, r.y);
    }
    // reduce lanes that share j (xor offsets >= B keep j fixed)
    double v[5] = {d_rr.get(), d_ri.get(), d_gr.get(), d_gi.get(), d_n.get()};
#pragma unroll
    for (int d = 0; d < 5; ++d)
        for (int o = 16; o >= B; o >>= 1) v[d] += __shfl_xor_sync(0xffffffffu, v[d], o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane < B) {
#pragma unroll
        for (int d = 0; d < 5; ++d) red[(warp * B + lane) * FTK_UPD_DOTS + d] = v[d];
    }
    __syncthreads();
    double *part = ua.partials + (size_t)blockIdx.x * B * FTK_UPD_DOTS;
    for (int q = threadIdx.x; q < B * FTK_UPD_DOTS; q += blockDim.x) {
        double s = 0.0;
        if (q % FTK_UPD_DOTS < 5)
            for (int ww = 0; ww < nw; ++ww) s += red[ww * B * FTK_UPD_DOTS + q];
        part[q] = s;
    }
    // last block: fixed-order sum of all partials -> ua.result[B][FTK_UPD_DOTS]
    __shared__ int am_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) am_last = (atomicAdd(ua.counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    for (int q = threadIdx.x; q < B * FTK_UPD_DOTS; q += blockDim.x) {
        double s = 0.0;
        for (int bb = 0; bb < (int)gridDim.x; ++bb)
            s += __ldcg(ua.partials + (size_t)bb * B * FTK_UPD_DOTS + q);
        ua.result[q] = s;
    }
    if (threadIdx.x == 0) *ua.counter = 0u;
}

// ------------------------------------------------------------ seed scalars
// One thread per RHS. Reads rho_k, g_k, |r_k| (update kernel) and
// mu_k = r_k^T H r_k (H pass), the max over shifts of 1/|pi_k| (shift
// kernel of the previous iteration), and computes
//   converged?  ||r_k|| max_s 1/|pi^s_k| <= tol ||lambda||   (k >= 1)
//   beta_{k-1} = rho_k / rho_{k-1}
//   alpha_k    = rho_k / (z_s rho_k - mu_k - beta_{k-1} rho_k / alpha_{k-1})
//   c_k        = beta_{k-1} alpha_k / alpha_{k-1}
// (the 3-term form of COCG on A = z_s - H; Sec. II.B).
__device__ void seed_one(const SeedArgs &sa, CocgSeed &s, int j);
__device__ __forceinline__ dcx cmul(dcx a, dcx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ dcx cdiv(dcx a, dcx b) {
    // Smith's algorithm
    if (fabs(b.re) >= fabs(b.im)) {
        double r = b.im / b.re, d = b.re + b.im * r;
        return {(a.re + a.im * r) / d, (a.im - a.re * r) / d};
    }
    double r = b.re / b.im, d = b.re * r + b.im;
    return {(a.re * r + a.im) / d, (a.im * r - a.re) / d};
}
__device__ __forceinline__ double cabs_(dcx a) { return hypot(a.re, a.im); }

__global__ void cocg_seed_kernel(SeedArgs sa) {
    const int j = threadIdx.x;
    if (j < sa.n_rhs) {
        CocgSeed &s = sa.seed[j];
        if (!s.done) seed_one(sa, s, j);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int all = 1;
        for (int q = 0; q < sa.n_rhs; ++q) all &= (sa.seed[q].done != 0);
        *sa.all_done = all;
    }
}

__device__ void seed_one(const SeedArgs &sa, CocgSeed &s, int j) {
    const double *ud = sa.upd + j * FTK_UPD_DOTS;
    const double *hd = sa.hv + j * FTK_HV_DOTS;
    dcx rho = {ud[0], ud[1]}, g = {ud[2], ud[3]}, mu = {hd[0], hd[1]};
    const double nrm = sqrt(fmax(ud[4], 0.0));
    const int k = s.k;
    if (k == 0) s.lnorm = nrm;
    // the shift kernel of iteration k-1 wrote max 1/|pi_k| into parity k;
    // clear parity k+1 for the shift kernel of this iteration
    const double inv_pi_max = sa.inv_pi_max[(k & 1) * FTK_MAX_RHS + j];
    sa.inv_pi_max[((k + 1) & 1) * FTK_MAX_RHS + j] = 0.0;
    if (k >= 1) {
        const double worst = nrm * inv_pi_max;
        s.resid = worst / s.lnorm;
        if (worst <= sa.tol * s.lnorm) { s.done = 1; return; }
        if (k >= sa.max_iter) { s.done = 4; return; }
    }
    if (nrm == 0.0 || cabs_(rho) <= 1e-300 * (nrm * nrm) || s.lnorm == 0.0) {
        s.done = (s.lnorm == 0.0 || nrm == 0.0) ? 1 : 2;
        return;
    }
    dcx zs = {s.zs_re, s.zs_im};
    dcx beta = {0, 0}, c = {0, 0};
    dcx denom = {cmul(zs, rho).re - mu.re, cmul(zs, rho).im - mu.im};
    if (k >= 1) {
        dcx rp = {s.rho_re, s.rho_im}, ap = {s.alpha_re, s.alpha_im};
        beta = cdiv(rho, rp);
        dcx t = cdiv(cmul(beta, rho), ap);
        denom.re -= t.re; denom.im -= t.im;
    }
    if (cabs_(denom) == 0.0) { s.done = 2; return; }
    dcx alpha = cdiv(rho, denom);
    if (k >= 1) {
        dcx ap = {s.alpha_re, s.alpha_im};
        c = cdiv(cmul(beta, alpha), ap);
    }
    s.rho_prev_re = s.rho_re; s.rho_prev_im = s.rho_im;
    s.rho_re = rho.re; s.rho_im = rho.im;
    s.alpha_prev_re = s.alpha_re; s.alpha_prev_im = s.alpha_im;
    s.alpha_re = alpha.re; s.alpha_im = alpha.im;
    s.beta_prev_re = beta.re; s.beta_prev_im = beta.im;
    s.c_re = c.re; s.c_im = c.im;
    s.g_re = g.re; s.g_im = g.im;
    s.nrm = nrm;
    s.k = k + 1;
    s.iters = k + 1;
}

// ------------------------------------------------------------ shift recurrences
// One thread per (shift, RHS). With D = z_s' - z_s (Frommer 2003):
//   beta^s_{k-1} = (pi_{k-1}/pi_k)^2 beta_{k-1}
//   p~^s_k       = g_k / pi_k + beta^s_{k-1} p~^s_{k-1}      (p~ = lambda^dag p^s)
//   pi_{k+1}     = (1 + alpha_k D) pi_k + c_k (pi_k - pi_{k-1})
//   alpha^s_k    = alpha_k pi_k / pi_{k+1},   G^s += alpha^s_k p~^s_k
// and the per-RHS max of 1/|pi_{k+1}| for the next convergence test.
__global__ void cocg_shift_kernel(ShiftArgs sh) {
    const int j = blockIdx.y;
    const int si = blockIdx.x * blockDim.x + threadIdx.x;
    const CocgSeed &s = sh.seed[j];
    __shared__ double wmax[256 / 32];
    double inv_pi = 0.0;
    bool active = (si < sh.n_omega) && !s.done;
    const size_t o = (size_t)j * sh.n_omega + si;
    if (active && sh.frozen[o]) active = false;
    if (active) {
        // freeze a shift whose residual ||r_k|| / |pi_k| reached tol ||lambda||
        const dcx pc0 = sh.pi_cur[o];
        if (s.nrm <= sh.tol * s.lnorm * cabs_(pc0)) { sh.frozen[o] = 1; active = false; }
    }
    if (active) {
        const int k = s.k - 1;   // iteration just computed by the seed kernel
        dcx pc = sh.pi_cur[o], pp = sh.pi_prev[o], pt = sh.ptil[o], G = sh.G[o];
        const dcx alpha = {s.alpha_re, s.alpha_im}, c = {s.c_re, s.c_im};
        const dcx beta = {s.beta_prev_re, s.beta_prev_im}, g = {s.g_re, s.g_im};
        const dcx D = {sh.omega[si] - sh.omega[sh.seed_idx], 0.0};
        dcx bs = {0, 0};
        if (k >= 1) { dcx r = cdiv(pp, pc); bs = cmul(cmul(r, r), beta); }
        dcx gp = cdiv(g, pc), bp = cmul(bs, pt);
        pt = {gp.re + bp.re, gp.im + bp.im};
        dcx aD = cmul(alpha, D);
        dcx t1 = cmul({1.0 + aD.re, aD.im}, pc);
        dcx t2 = cmul(c, {pc.re - pp.re, pc.im - pp.im});
        dcx pn = {t1.re + t2.re, t1.im + t2.im};
        dcx as = cdiv(cmul(alpha, pc), pn);
        dcx ag = cmul(as, pt);
        G.re += ag.re; G.im += ag.im;
        sh.pi_prev[o] = pc; sh.pi_cur[o] = pn; sh.ptil[o] = pt; sh.G[o] = G;
        inv_pi = 1.0 / cabs_(pn);
    }
    // block max -> atomicMax on the (non-negative) double's bit pattern
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) inv_pi = fmax(inv_pi, __shfl_xor_sync(0xffffffffu, inv_pi, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = inv_pi;
    __syncthreads();
    if (threadIdx.x == 0 && !s.done) {
        double m = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, wmax[w]);
        atomicMax(reinterpret_cast<unsigned long long *>(sh.inv_pi_max + ((s.k & 1) * FTK_MAX_RHS) + j),
                  (unsigned long long)__double_as_longlong(m));
    }
}

// ------------------------------------------------------------ probe S^gamma_q
// lambda = s N^{-1/2} sum_l exp(i q.R_l) S^gamma_l psi   (Sec. V)
//   gamma = z: lambda[x] = s psi[x] sum_l f_l s_l(x)/2
//   gamma = x: lambda[x] = s sum_l f_l psi[x ^ 2^l] / 2
//   gamma = y: lambda[x] = s sum_l f_l (-i s_l(x)/2) psi[x ^ 2^l]
// (S^y|x> = (i s_l(x)/2)|x ^ 2^l> read from the source x ^ 2^l.)
// Fused: ||lambda||^2 (last-block reduction).
template <typename R>
__global__ void __launch_bounds__(256)
apply_op_kernel(const typename C2<R>::t *__restrict__ psi, typename C2<R>::t *lam, OpArgs oa) {
    typedef typename C2<R>::t cx;
    __shared__ double red[(256 / 32) * 1];
    __shared__ double fr[FTK_MAX_SITES], fi[FTK_MAX_SITES];
    if (threadIdx.x < oa.n_sites) { fr[threadIdx.x] = oa.f_re[threadIdx.x]; fi[threadIdx.x] = oa.f_im[threadIdx.x]; }
    __syncthreads();
    const double sc = *oa.scale;
    Acc<double> nrm;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < oa.dim;
         x += (uint64_t)gridDim.x * blockDim.x) {
        double re = 0, im = 0;
        if (oa.gamma == 2) {
            double fre = 0, fim = 0;
            for (int l = 0; l < oa.n_sites; ++l) {
                const double s = ((x >> l) & 1) ? 0.5 : -0.5;
                fre += s * fr[l]; fim += s * fi[l];
            }
            const cx p = psi[x];
            re = fre * (double)p.x - fim * (double)p.y;
            im = fre * (double)p.y + fim * (double)p.x;
        } else {
            for (int l = 0; l < oa.n_sites; ++l) {
                const cx p = psi[x ^ (1ull << l)];
                double ar = fr[l] * 0.5, ai = fi[l] * 0.5;
                if (oa.gamma == 1) {   // times -i s_l(x)
                    const double s = ((x >> l) & 1) ? 1.0 : -1.0;
                    const double tr = ai * s, ti = -ar * s;
                    ar = tr; ai = ti;
                }
                re += ar * (double)p.x - ai * (double)p.y;
                im += ar * (double)p.y + ai * (double)p.x;
            }
        }
        re *= sc; im *= sc;
        const R rr = (R)re, ri = (R)im;
        lam[x] = mk<R>(rr, ri);
        nrm.add((double)rr * (double)rr + (double)ri * (double)ri);
    }
    double v[1] = {nrm.get()};
    block_reduce<1>(v, red);
    if (threadIdx.x == 0) oa.partials[blockIdx.x] = red[0];
    if (!last_block_reduce<1>(oa.partials, oa.counter, oa.result, red)) return;
    if (threadIdx.x == 0) {
        oa.slot_energy[0] = oa.energy_src ? *oa.energy_src * oa.n_sites_d : oa.energy_val;
        oa.slot_norm2[0] = oa.result[0];
    }
}

// ------------------------------------------------------------ random state
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): round
//   (c0,c1,c2,c3) -> (hi(M1 c2)^c1^k0, lo(M1 c2), hi(M0 c0)^c3^k1, lo(M0 c0)),
// M0 = 0xD2511F53, M1 = 0xCD9E8D57, key bump (0x9E3779B9, 0xBB67AE85).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u; k.y += 0xBB67AE85u;
    }
    return c;
}

template <typename R>
__global__ void __launch_bounds__(256)
init_state_kernel(typename C2<R>::t *v, InitArgs ia) {
    __shared__ double red[(256 / 32) * 1];
    const uint2 key = make_uint2((uint32_t)ia.seed, (uint32_t)(ia.seed >> 32));
    Acc<double> nrm;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < ia.dim;
         x += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)x, (uint32_t)(x >> 32), ia.sample, 0u), key);
        const double u1 = ((double)((((uint64_t)w.x << 32) | w.y) >> 11) + 0.5) * 0x1p-53;
        const double u2 = ((double)((((uint64_t)w.z << 32) | w.w) >> 11) + 0.5) * 0x1p-53;
        const double rad = sqrt(-2.0 * log(u1));
        double sn, cs;
        sincospi(2.0 * u2, &sn, &cs);
        const R re = (R)(rad * cs), im = (R)(rad * sn);
        v[x] = mk<R>(re, im);
        nrm.add((double)re * (double)re + (double)im * (double)im);
    }
    double vv[1] = {nrm.get()};
    block_reduce<1>(vv, red);
    if (threadIdx.x == 0) ia.partials[blockIdx.x] = red[0];
    if (!last_block_reduce<1>(ia.partials, ia.counter, ia.result, red)) return;
    if (threadIdx.x == 0) {
        ia.tpq->scale = 1.0 / sqrt(ia.result[0]);
        ia.tpq->logQ = 0.0;
        ia.tpq->k = 0;
    }
}

// norm of a vector -> tpq scale (ftk_set_state)
template <typename R>
__global__ void __launch_bounds__(256)
norm_kernel(const typename C2<R>::t *v, InitArgs ia) {
    typedef typename C2<R>::t cx;
    __shared__ double red[(256 / 32) * 1];
    Acc<double> nrm;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < ia.dim;
         x += (uint64_t)gridDim.x * blockDim.x) {
        const cx p = v[x];
        nrm.add((double)p.x * (double)p.x + (double)p.y * (double)p.y);
    }
    double vv[1] = {nrm.get()};
    block_reduce<1>(vv, red);
    if (threadIdx.x == 0) ia.partials[blockIdx.x] = red[0];
    if (!last_block_reduce<1>(ia.partials, ia.counter, ia.result, red)) return;
    if (threadIdx.x == 0 && ia.tpq) {
        ia.tpq->scale = 1.0 / sqrt(ia.result[0]);
        ia.tpq->logQ = 0.0;
        ia.tpq->k = 0;
    }
}

// double (re, im) <-> context precision, with an optional device scale
template <typename R>
__global__ void convert_in_kernel(const double2 *src, typename C2<R>::t *dst, uint64_t n) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const double2 s = src[i];
        dst[i] = mk<R>((R)s.x, (R)s.y);
    }
}

template <typename R>
__global__ void convert_out_kernel(const typename C2<R>::t *src, double2 *dst, uint64_t n,
                                   const double *scale) {
    const double sc = scale ? *scale : 1.0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const typename C2<R>::t s = src[i];
        dst[i] = make_double2(sc * (double)s.x, sc * (double)s.y);
    }
}

// ------------------------------------------------------------ spectrum
// One CTA per temperature. Weights (reading R1 of Eq. B1):
//   log w_2k   = 2k log(N beta) - lgamma(2k+1) + 2 log Q_k
//   log w_2k+1 = (2k+1) log(N beta) - lgamma(2k+2) + 2 log Q_k + log(l - u_k)
// W_s = sum of w_n with round(floor(n/2)/se) == s (ties up), normalised by
// log-sum-exp; S(w) = sum_s W_s (-Im G_s(w) / pi).
__global__ void __launch_bounds__(256) spectrum_kernel(SpecArgs sp) {
    __shared__ double red[(256 / 32) * 1];
    __shared__ double wsh[1024];
    const int t = blockIdx.x;
    const double beta = 1.0 / sp.T[t];
    const double lnb = log(sp.n_sites * beta);
    const int K = sp.n_steps, nterm = 2 * K;
    // pass 1: max log-weight
    double m = -INFINITY;
    for (int n = threadIdx.x; n < nterm; n += blockDim.x) {
        const int k = n >> 1;
        double lw = n * lnb - lgamma((double)n + 1.0) + 2.0 * sp.logq[k];
        if (n & 1) lw += log(sp.ell - sp.u[k]);
        m = fmax(m, lw);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double mm = -INFINITY;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = fmax(mm, red[w]);
        red[0] = mm;
    }
    __syncthreads();
    const double mx = red[0];
    __syncthreads();
    // pass 2: per-shell sums (shells processed by thread groups, fixed order)
    for (int s = threadIdx.x; s < sp.n_shell; s += blockDim.x) wsh[s] = 0.0;
    __syncthreads();
    const int se = sp.save_every;
    for (int s = threadIdx.x; s < sp.n_shell; s += blockDim.x) {
        // steps k mapped to shell s: round(k/se) == s (ties up) and k < K
        // floor(k/se + 1/2) == s  <=>  s se - floor(se/2) <= k <= s se + floor((se-1)/2)
        int k_lo = s * se - se / 2;
        int k_hi = s * se + (se - 1) / 2;
        if (k_lo < 0) k_lo = 0;
        if (s == sp.n_shell - 1) k_hi = K - 1;
        if (k_hi > K - 1) k_hi = K - 1;
        double acc = 0.0;
        for (int k = k_lo; k <= k_hi; ++k) {
            for (int par = 0; par < 2; ++par) {
                const int n = 2 * k + par;
                double lw = n * lnb - lgamma((double)n + 1.0) + 2.0 * sp.logq[k];
                if (par) lw += log(sp.ell - sp.u[k]);
                acc += exp(lw - mx);
            }
        }
        wsh[s] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int s = 0; s < sp.n_shell; ++s) tot += wsh[s];
        red[0] = tot;
        // truncation: tail w_{2K-1} r/(1-r), r = N beta (l - u_{K-1}) / (2K)
        const int kk = K - 1;
        const double r = sp.n_sites * beta * (sp.ell - sp.u[kk]) / (2.0 * kk + 2.0);
        double lw = (2.0 * kk + 1) * lnb - lgamma(2.0 * kk + 2.0) + 2.0 * sp.logq[kk] + log(sp.ell - sp.u[kk]);
        int tr = 1;
        if (r < 1.0) tr = (exp(lw - mx) * r / (1.0 - r) > 1e-14 * tot) ? 1 : 0;
        sp.trunc[t] = tr;
    }
    __syncthreads();
    const double tot = red[0];
    for (int w = threadIdx.x; w < sp.n_omega; w += blockDim.x) {
        double acc = 0.0;
        for (int s = 0; s < sp.n_shell; ++s)
            acc += wsh[s] * (-sp.G[2 * ((size_t)s * sp.n_omega + w) + 1] / M_PI);
        sp.S[(size_t)t * sp.n_omega + w] = acc / tot;
    }
}

// ================================================================ launchers
template <typename R, int B>
static cudaError_t hv_dispatch_epi(int epi, const void *in, void *out, const PassDesc &pd,
                                   const EpiArgs &ea, int grid, int threads, size_t smem,
                                   cudaStream_t st) {
    typedef typename C2<R>::t cx;
    void (*k)(const cx *, cx *, const PassDesc, const EpiArgs) = nullptr;
    if (epi == EPI_PLAIN) k = hv_pass_kernel<R, B, EPI_PLAIN>;
    else if (epi == EPI_COCG) k = hv_pass_kernel<R, B, EPI_COCG>;
    else if (epi == EPI_TPQ) {
        if (B != 1) return cudaErrorInvalidValue;
        k = hv_pass_kernel<R, 1, EPI_TPQ>;
    }
    if (!k) return cudaErrorInvalidValue;
    k<<<grid, threads, smem, st>>>(reinterpret_cast<const cx *>(in), reinterpret_cast<cx *>(out), pd, ea);
    return cudaGetLastError();
}

template <typename R>
static cudaError_t hv_dispatch_b(int B, int epi, const void *in, void *out, const PassDesc &pd,
                                 const EpiArgs &ea, int grid, int threads, size_t smem, cudaStream_t st) {
    switch (B) {
    case 1: return hv_dispatch_epi<R, 1>(epi, in, out, pd, ea, grid, threads, smem, st);
    case 2: return hv_dispatch_epi<R, 2>(epi, in, out, pd, ea, grid, threads, smem, st);
    case 4: return hv_dispatch_epi<R, 4>(epi, in, out, pd, ea, grid, threads, smem, st);
    case 8: return hv_dispatch_epi<R, 8>(epi, in, out, pd, ea, grid, threads, smem, st);
    case 16: return hv_dispatch_epi<R, 16>(epi, in, out, pd, ea, grid, threads, smem, st);
    case 32: return hv_dispatch_epi<R, 32>(epi, in, out, pd, ea, grid, threads, smem, st);
    default: return cudaErrorInvalidValue;
    }
}

// Opt every H.V pass instantiation into the full 227 KB of shared memory
// once per process (must happen outside stream capture).
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

template <typename R, int B>
static cudaError_t attrs_b() {
    cudaError_t e = opt_in(hv_pass_kernel<R, B, EPI_PLAIN>);
    if (e == cudaSuccess) e = opt_in(hv_pass_kernel<R, B, EPI_COCG>);
    if (e == cudaSuccess && B == 1) e = opt_in(hv_pass_kernel<R, 1, EPI_TPQ>);
    return e;
}

cudaError_t init_kernel_attributes() {
    static int done = 0;
    static cudaError_t status = cudaSuccess;
    if (done) return status;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = attrs_b<double, 1>();
    if (e == cudaSuccess) e = attrs_b<double, 2>();
    if (e == cudaSuccess) e = attrs_b<double, 4>();
    if (e == cudaSuccess) e = attrs_b<double, 8>();
    if (e == cudaSuccess) e = attrs_b<double, 16>();
    if (e == cudaSuccess) e = attrs_b<double, 32>();
    if (e == cudaSuccess) e = attrs_b<float, 1>();
    if (e == cudaSuccess) e = attrs_b<float, 2>();
    if (e == cudaSuccess) e = attrs_b<float, 4>();
    if (e == cudaSuccess) e = attrs_b<float, 8>();
    if (e == cudaSuccess) e = attrs_b<float, 16>();
    if (e == cudaSuccess) e = attrs_b<float, 32>();
    status = e;
    done = 1;
    return e;
}

cudaError_t launch_hv_pass(int prec, int B, int epi, const void *in, void *out, const PassDesc &pd,
                           const EpiArgs &ea, int grid, int threads, size_t smem, cudaStream_t st) {
    if (prec == 0) return hv_dispatch_b<double>(B, epi, in, out, pd, ea, grid, threads, smem, st);
    return hv_dispatch_b<float>(B, epi, in, out, pd, ea, grid, threads, smem, st);
}

size_t hv_smem_bytes(int prec, int B, int tile_bits, int chunk_bits, int threads) {
    const size_t elem = prec == 0 ? 16 : 8;
    const size_t n_hi = (size_t)1 << (tile_bits - chunk_bits);
    const int nd = 2 * B > 2 ? 2 * B : 2;
    return ((size_t)1 << tile_bits) * B * elem + (n_hi + (n_hi & 1)) * 4 + (size_t)(threads / 32) * nd * 8;
}

template <typename R>
static cudaError_t upd_dispatch(int B, const void *rcur, const void *w, void *rprev_new,
                                const UpdArgs &ua, int grid, cudaStream_t st) {
    typedef typename C2<R>::t cx;
#define FTK_UPD_CASE(BB)                                                                     \
    case BB:                                                                                 \
        cocg_update_kernel<R, BB><<<grid, 256, 0, st>>>(reinterpret_cast<const cx *>(rcur), \
            reinterpret_cast<const cx *>(w), reinterpret_cast<cx *>(rprev_new), ua);         \
        break;
    switch (B) {
        FTK_UPD_CASE(1) FTK_UPD_CASE(2) FTK_UPD_CASE(4) FTK_UPD_CASE(8) FTK_UPD_CASE(16) FTK_UPD_CASE(32)
    default: return cudaErrorInvalidValue;
    }
#undef FTK_UPD_CASE
    return cudaGetLastError();
}

cudaError_t launch_cocg_update(int prec, int B, const void *rcur, const void *w, void *rprev_new,
                               const UpdArgs &ua, int grid, cudaStream_t st) {
    if (prec == 0) return upd_dispatch<double>(B, rcur, w, rprev_new, ua, grid, st);
    return upd_dispatch<float>(B, rcur, w, rprev_new, ua, grid, st);
}

cudaError_t launch_cocg_seed(const SeedArgs &sa, cudaStream_t st) {
    cocg_seed_kernel<<<1, 32, 0, st>>>(sa);
    return cudaGetLastError();
}

cudaError_t launch_cocg_shift(const ShiftArgs &sh, int n_rhs, cudaStream_t st) {
    dim3 grid((sh.n_omega + 255) / 256, n_rhs);
    cocg_shift_kernel<<<grid, 256, 0, st>>>(sh);
    return cudaGetLastError();
}

cudaError_t launch_apply_op(int prec, const void *psi, void *lam, const OpArgs &oa, int grid,
                            cudaStream_t st) {
    if (prec == 0)
        apply_op_kernel<double><<<grid, 256, 0, st>>>(reinterpret_cast<const double2 *>(psi),
                                                      reinterpret_cast<double2 *>(lam), oa);
    else
        apply_op_kernel<float><<<grid, 256, 0, st>>>(reinterpret_cast<const float2 *>(psi),
                                                     reinterpret_cast<float2 *>(lam), oa);
    return cudaGetLastError();
}

cudaError_t launch_init_state(int prec, void *v, const InitArgs &ia, int grid, cudaStream_t st) {
    if (prec == 0) init_state_kernel<double><<<grid, 256, 0, st>>>(reinterpret_cast<double2 *>(v), ia);
    else init_state_kernel<float><<<grid, 256, 0, st>>>(reinterpret_cast<float2 *>(v), ia);
    return cudaGetLastError();
}

cudaError_t launch_norm(int prec, const void *v, const InitArgs &ia, int grid, cudaStream_t st) {
    if (prec == 0) norm_kernel<double><<<grid, 256, 0, st>>>(reinterpret_cast<const double2 *>(v), ia);
    else norm_kernel<float><<<grid, 256, 0, st>>>(reinterpret_cast<const float2 *>(v), ia);
    return cudaGetLastError();
}

cudaError_t launch_convert_in(int prec, const void *src, void *dst, uint64_t n, int grid, cudaStream_t st) {
    if (prec == 0) convert_in_kernel<double><<<grid, 256, 0, st>>>(reinterpret_cast<const double2 *>(src), reinterpret_cast<double2 *>(dst), n);
    else convert_in_kernel<float><<<grid, 256, 0, st>>>(reinterpret_cast<const double2 *>(src), reinterpret_cast<float2 *>(dst), n);
    return cudaGetLastError();
}

cudaError_t launch_convert_out(int prec, const void *src, void *dst, uint64_t n, const double *scale,
                               int grid, cudaStream_t st) {
    if (prec == 0) convert_out_kernel<double><<<grid, 256, 0, st>>>(reinterpret_cast<const double2 *>(src), reinterpret_cast<double2 *>(dst), n, scale);
    else convert_out_kernel<float><<<grid, 256, 0, st>>>(reinterpret_cast<const float2 *>(src), reinterpret_cast<double2 *>(dst), n, scale);
    return cudaGetLastError();
}

cudaError_t launch_spectrum(const SpecArgs &sp, int n_T, cudaStream_t st) {
    spectrum_kernel<<<n_T, 256, 0, st>>>(sp);
    return cudaGetLastError();
}

}  // namespace ftk
