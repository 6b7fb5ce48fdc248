// CUDA kernels of the FTKomega hot path (sm_103a). No tensor cores: the
// Hamiltonian-vector product is a bit-indexed gather, not a contraction.
//
//   (the H.V pass lives in ftk_hv.cu)
//   cocg_update 3-term seed-COCG residual update with fused dots (Sec. II.B);
//               cocg_update_df_kernel: the same on float hi + lo pairs (mixed
//               and double-float modes; the double-float solve runs it only
//               for its first step and in the relaxed phase, its other steps
//               update inside the first H.V pass)
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
#include "ftk_device.cuh"
#include "ftk_kernels.h"

#include <math.h>

namespace ftk {

// --------------------------------------------------------- COCG update
// Block vectors are stored RHS by RHS: element (x, j) at j * dim + x.
// Grid (gx, B): blockIdx.y = j.
// mode 0: r_0 = lambda_j (start);  mode 1: 3-term seed residual update
//   r_{k+1} = (1 + c_k) r_k - alpha_k (z_s r_k - w_k) - c_k r_{k-1}
// evaluated as r_k + c_k (r_k - r_{k-1}) - alpha_k (z_s r_k - w_k) and written
// over r_{k-1}. z_s r - w is formed by FMAs from a hi + lo split of z_s
// (exact products, one rounding of the small difference), so FP32 vectors
// lose no digits to the cancellation between z_s r and H r. Fused dots of
// r_{k+1}: rho = r^T r, g = lambda^dag r, |r|^2 (FTK_UPD_DOTS doubles per RHS).
// A finished RHS (done != 0) is skipped; its block contributes zeros.
//
// PlainVec: R vectors and R arithmetic (FP64 and FP32 modes; the mixed mode
// has its own kernel below).
template <typename R>
struct PlainVec {
    typedef typename C2<R>::t cx;
    typedef R A;   // arithmetic type
    cx *rcur;
    const cx *w;
    cx *rnew;
    __device__ cx load_r(size_t i) const { return rcur[i]; }
    __device__ cx load_rp(size_t i) const { return rnew[i]; }
    __device__ cx load_w(size_t i) const { return w[i]; }
    __device__ void store(size_t i, cx r) const { rnew[i] = r; }
    __device__ void store_cur(size_t i, cx r) const { rcur[i] = r; }
};
template <typename V>
__global__ void __launch_bounds__(256) cocg_update_kernel(V vec, UpdArgs ua) {
    typedef typename V::A R;
    typedef typename C2<R>::t cx;
    __shared__ double red[(256 / 32) * 5];
    if (*ua.all_done) return;
    const int j = blockIdx.y;
    const uint64_t n = ua.dim;
    const size_t off = (size_t)j * n;
    const bool skip = ua.mode == 1 && ua.seed[j].done != 0;
    R zr_hi = 0, zr_lo = 0, zi_hi = 0, zi_lo = 0, al_re = 0, al_im = 0, c_re = 0, c_im = 0;
    if (ua.mode == 1) {
        const CocgSeed &s = ua.seed[j];
        zr_hi = (R)s.zs_re; zr_lo = (R)(s.zs_re - (double)zr_hi);
        zi_hi = (R)s.zs_im; zi_lo = (R)(s.zs_im - (double)zi_hi);
        al_re = (R)s.alpha_re; al_im = (R)s.alpha_im;
        c_re = (R)s.c_re; c_im = (R)s.c_im;
    }
    const cx *lam = reinterpret_cast<const cx *>(ua.lambda[j]);
    // g = proj^dag r: the projection vector (A of <A|(z - H)^-1|B>), lambda by default
    const cx *prj = ua.proj[j] ? reinterpret_cast<const cx *>(ua.proj[j]) : lam;
    // range guard of the seed kernel: r_{k+1} and r_k (the next r_{k-1}) scaled by f
    const R f = ua.mode == 1 ? (R)ua.seed[j].rescale : (R)1;
    Acc<R> d_rr, d_ri, d_gr, d_gi, d_n;
    if (!skip) {
        for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
             x += (uint64_t)gridDim.x * blockDim.x) {
            const cx l = prj[x];
            cx r;
            if (ua.mode == 0) {
                r = lam[x];
            } else {
                const cx rc = vec.load_r(off + x), wc = vec.load_w(off + x), rp = vec.load_rp(off + x);
                // A r = z_s r - w (the lo terms of z_s vanish in double)
                R ar = fma(zr_hi, rc.x, -wc.x);
                ar = fma(-zi_hi, rc.y, ar);
                R ai = fma(zr_hi, rc.y, -wc.y);
                ai = fma(zi_hi, rc.x, ai);
                if constexpr (sizeof(R) == 4) {
                    ar = fma(zr_lo, rc.x, ar);
                    ar = fma(-zi_lo, rc.y, ar);
                    ai = fma(zr_lo, rc.y, ai);
                    ai = fma(zi_lo, rc.x, ai);
                }
                // d = c (r - r_prev) - alpha A r
                const R tr = rc.x - rp.x, ti = rc.y - rp.y;
                R dr = c_re * tr - c_im * ti;
                R di = c_re * ti + c_im * tr;
                dr = fma(-al_re, ar, dr); dr = fma(al_im, ai, dr);
                di = fma(-al_re, ai, di); di = fma(-al_im, ar, di);
                r = mk<R>(rc.x + dr, rc.y + di);
                if (f != (R)1) {
                    r = mk<R>(r.x * f, r.y * f);
                    vec.store_cur(off + x, mk<R>(rc.x * f, rc.y * f));
                }
            }
            vec.store(off + x, r);
            d_rr.fma2(r.x, r.x); d_rr.fma2(-r.y, r.y);
            d_ri.fma2(2 * r.x, r.y);
            d_gr.fma2(l.x, r.x); d_gr.fma2(l.y, r.y);
            d_gi.fma2(l.x, r.y); d_gi.fma2(-l.y, r.x);
            d_n.fma2(r.x, r.x); d_n.fma2(r.y, r.y);
        }
    }
    double v[5] = {d_rr.get(), d_ri.get(), d_gr.get(), d_gi.get(), d_n.get()};
    block_reduce<5>(v, red);
    const unsigned nblk = gridDim.x * gridDim.y;
    double *part = ua.partials + ((size_t)j * gridDim.x + blockIdx.x) * 5;
    if (threadIdx.x < 5) part[threadIdx.x] = red[threadIdx.x];
    // last block: fixed-order sum of the partials -> ua.result[B][FTK_UPD_DOTS]
    __shared__ int am_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) am_last = (atomicAdd(ua.counter, 1u) == nblk - 1);
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    for (int q = threadIdx.x; q < (int)gridDim.y * 5; q += blockDim.x) {
        const int jj = q / 5, d = q % 5;
        double sum = 0.0;
        for (unsigned bb = 0; bb < gridDim.x; ++bb)
            sum += __ldcg(ua.partials + ((size_t)jj * gridDim.x + bb) * 5 + d);
        ua.result[jj * FTK_UPD_DOTS + d] = sum;
    }
    if (threadIdx.x == 0) *ua.counter = 0u;
}

// Mixed and double-float modes: the residuals r_k, r_{k-1} (float hi + lo
// pairs, lo ua.lo_stride float2 after hi; w is float, or a pair with its lo
// ua.w_lo float2 after hi in the double-float mode) are updated in double-float
// arithmetic on the FP32 pipe (about 48 bits, the precision of the stored
// pairs). The dots rho = r^T r and g = lambda^dag r accumulate the exact FMA
// two-products of the hi parts plus the hi x lo cross terms with two-sums
// (double-float, ~48 bits; the FP64 pipe is not used in the element loop);
// |r|^2 (the convergence test) uses the hi parts with compensated float
// accumulation. Mode 0 splits the FP64 lambda once into float hi + lo
// (ua.lam_split), which the iterations read.
__global__ void __launch_bounds__(256)
cocg_update_df_kernel(float2 *rcur, const float2 *__restrict__ w, float2 *rnew, UpdArgs ua) {
    __shared__ double red[(256 / 32) * 5];
    if (*ua.all_done) return;
    if (ua.lowp && *ua.lowp != ua.lowp_run) return;
    const int j = blockIdx.y;
    const uint64_t n = ua.dim;
    const size_t off = (size_t)j * n;
    const long long lo = ua.lo_stride;
    const bool skip = ua.mode == 1 && ua.seed[j].done != 0;
    DfStep q{};
    if (ua.mode == 1) q = df_step(ua.seed[j]);   // range guard: q.f is a power of two
    const double2 *lam = reinterpret_cast<const double2 *>(ua.lambda[j]);
    float4 *lsp = ua.lam_split + off;
    DfUpdDots dots;
    if (!skip) {
        for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
             x += (uint64_t)gridDim.x * blockDim.x) {
            float4 l4;
            dcl r;
            const size_t i = off + x;
            if (ua.mode == 0) {
                const double2 ld = lam[x];
                r = {dfl_from(ld.x), dfl_from(ld.y)};
                // the projection vector's split (lambda's unless another is given)
                const double2 pv = ua.proj[j] ? reinterpret_cast<const double2 *>(ua.proj[j])[x] : ld;
                const dfl pr = dfl_from(pv.x), pim = dfl_from(pv.y);
                l4 = make_float4(pr.hi, pim.hi, pr.lo, pim.lo);
                lsp[x] = l4;
            } else {
                l4 = lsp[x];
                const float2 ch = rcur[i], cl = rcur[i + lo], ph = rnew[i], pl = rnew[i + lo], wv = w[i];
                const float2 wl = ua.w_lo ? w[i + ua.w_lo] : make_float2(0.f, 0.f);   // double-float w
                r = df_next_residual({{ch.x, cl.x}, {ch.y, cl.y}}, {{ph.x, pl.x}, {ph.y, pl.y}},
                                     {{wv.x, wl.x}, {wv.y, wl.y}}, q);
                if (q.f != 1.f) {
                    rcur[i] = make_float2(ch.x * q.f, ch.y * q.f);
                    rcur[i + lo] = make_float2(cl.x * q.f, cl.y * q.f);
                }
            }
            rnew[i] = make_float2(r.re.hi, r.im.hi);
            rnew[i + lo] = make_float2(r.re.lo, r.im.lo);
            dots.add(r, l4);
        }
    }
    double v[5];
    dots.get(v);
    block_reduce<5>(v, red);
    const unsigned nblk = gridDim.x * gridDim.y;
    double *part = ua.partials + ((size_t)j * gridDim.x + blockIdx.x) * 5;
    if (threadIdx.x < 5) part[threadIdx.x] = red[threadIdx.x];
    // last block: fixed-order sum of the partials -> ua.result[B][FTK_UPD_DOTS]
    __shared__ int am_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) am_last = (atomicAdd(ua.counter, 1u) == nblk - 1);
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    for (int q = threadIdx.x; q < (int)gridDim.y * 5; q += blockDim.x) {
        const int jj = q / 5, d = q % 5;
        double sum = 0.0;
        for (unsigned bb = 0; bb < gridDim.x; ++bb)
            sum += __ldcg(ua.partials + ((size_t)jj * gridDim.x + bb) * 5 + d);
        ua.result[jj * FTK_UPD_DOTS + d] = sum;
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
        s.sw = 0;
        if (!s.done) seed_one(sa, s, j);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int all = 1, small = 1;
        for (int q = 0; q < sa.n_rhs; ++q) {
            const CocgSeed &s = sa.seed[q];
            all &= (s.done != 0);
            if (!s.done) small &= (s.k >= 2 && s.resid < sa.relax);   // resid set from k = 1 on
        }
        *sa.all_done = all;
        // relaxed solve: from here on the matrix-vector products may run in
        // FP32 (their errors enter scaled by the small residual)
        if (sa.lowp && sa.relax > 0.0 && small && !all) *sa.lowp = 1;
    }
}

__device__ void seed_one(const SeedArgs &sa, CocgSeed &s, int j) {
    const double *ud = sa.upd + j * FTK_UPD_DOTS;
    const double *hd = sa.hv + j * FTK_HV_DOTS;
    dcx rho = {ud[0], ud[1]}, g = {ud[2], ud[3]}, mu = {hd[0], hd[1]};
    double nrm = sqrt(fmax(ud[4], 0.0));
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
    if (!isfinite(nrm) || !isfinite(rho.re) || !isfinite(rho.im) || !isfinite(mu.re) || !isfinite(mu.im)) {
        s.done = 5;   // non-finite residual or dots: breakdown
        return;
    }
    if (nrm == 0.0 || s.lnorm == 0.0) { s.done = 1; return; }     // exact solution
    if (sa.seed_switch && k >= 1 && nrm <= sa.tol * s.lnorm) {
        // Seed switching: the seed system has converged while other shifts
        // have not (else the test above would have stopped the solve). The
        // unconverged shift with the largest residual ||r_k|| / |pi^s_k|, i.e.
        // the smallest |pi^s_k|, becomes the seed. Only residuals enter the
        // recurrences, so with s1 = 1/pi*_k and s0 = 1/pi*_{k-1} the switch is
        // exact: r_k, w_k, g_k scale by s1, r_{k-1} by s0, rho_k and mu_k by
        // s1^2, rho_{k-1} by s0^2, alpha_{k-1} becomes the shift's
        // alpha*_{k-1} = alpha_{k-1} s1 / s0, and every pi^s_k, pi^s_{k-1} is
        // divided by pi*_k, pi*_{k-1} (the switch kernel scales the vectors
        // and the pi arrays); G, p~ and every shifted residual are unchanged.
        const dcx *pc = sa.pi_cur + (size_t)j * sa.n_omega;
        const dcx *pp = sa.pi_prev + (size_t)j * sa.n_omega;
        const int *fz = sa.frozen + (size_t)j * sa.n_omega;
        const double lim = nrm / (sa.tol * s.lnorm);   // unconverged: |pi| < lim
        int best = -1;
        double bmin = lim;
        for (int q = 0; q < sa.n_omega; ++q) {
            if (fz[q]) continue;
            const double a = cabs_(pc[q]);
            if (a < bmin) { bmin = a; best = q; }
        }
        if (best >= 0 && best != s.seed_idx) {
            const dcx one = {1.0, 0.0};
            const dcx s1 = cdiv(one, pc[best]), s0 = cdiv(one, pp[best]);
            const dcx s1s = cmul(s1, s1), s0s = cmul(s0, s0);
            rho = cmul(rho, s1s);
            mu = cmul(mu, s1s);
            g = cmul(g, s1);
            nrm *= cabs_(s1);
            const dcx rp = cmul({s.rho_re, s.rho_im}, s0s);
            s.rho_re = rp.re; s.rho_im = rp.im;
            const dcx ap = cmul({s.alpha_re, s.alpha_im}, cdiv(s1, s0));
            s.alpha_re = ap.re; s.alpha_im = ap.im;
            s.zs_re = s.e0 + sa.shift[best].re;
            s.zs_im = sa.shift[best].im;
            s.seed_idx = best;
            s.sw = 1;
            s.s1_re = s1.re; s.s1_im = s1.im; s.s0_re = s0.re; s.s0_im = s0.im;
            s.switches += 1;
        }
    }
    // r^T r vanished: at a residual 1e-12 below ||lambda|| this is the
    // underflow of FP32 vectors (the seed system is solved far beyond any
    // shifted one can still gain): stop as converged; otherwise a breakdown
    if (cabs_(rho) <= 1e-300 * (nrm * nrm)) { s.done = nrm <= 1e-12 * s.lnorm ? 1 : 2; return; }
    dcx zs = {s.zs_re, s.zs_im};
    dcx beta = {0, 0}, c = {0, 0};
    dcx denom = {cmul(zs, rho).re - mu.re, cmul(zs, rho).im - mu.im};
    if (k >= 1) {
        dcx rp = {s.rho_re, s.rho_im}, ap = {s.alpha_re, s.alpha_im};
        beta = cdiv(rho, rp);
        dcx t = cdiv(cmul(beta, rho), ap);
        denom.re -= t.re; denom.im -= t.im;
    }
    if (cabs_(denom) == 0.0) { s.done = 3; return; }
    dcx alpha = cdiv(rho, denom);
    if (k >= 1) {
        dcx ap = {s.alpha_re, s.alpha_im};
        c = cdiv(cmul(beta, alpha), ap);
    }
    // Range guard: the seed residual can fall many orders below ||lambda||
    // while slow shifts still converge (their |pi| falls with it); FP32 and
    // float-pair storage would underflow. Every quantity of the recurrences
    // is homogeneous in (r, pi), so r_k, r_{k+1} and all pi^s are scaled by
    // the same power of two f (exact), and the stored rho_k by f^2; the
    // shifted residuals r / pi^s, alpha, beta, c and G are unchanged.
    double f = 1.0;
    if (nrm < 0x1p-40 * s.lnorm) f = ldexp(1.0, ilogb(s.lnorm) - ilogb(nrm));
    s.rescale = f;
    s.rho_prev_re = s.rho_re; s.rho_prev_im = s.rho_im;
    s.rho_re = rho.re * f * f; s.rho_im = rho.im * f * f;
    s.alpha_prev_re = s.alpha_re; s.alpha_prev_im = s.alpha_im;
    s.alpha_re = alpha.re; s.alpha_im = alpha.im;
    s.beta_prev_re = beta.re; s.beta_prev_im = beta.im;
    s.c_re = c.re; s.c_im = c.im;
    const dcx az = cmul(alpha, zs);   // r_{k+1} = a1 r_k - c r_{k-1} + alpha w_k
    s.a1_re = 1.0 + c.re - az.re; s.a1_im = c.im - az.im;
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
    // history (right-hand side 0): iteration k = s.k - 1 of a running solve
    const int kh = s.k - 1;
    dcx* hrec = (sh.hist && j == 0 && !s.done && si < sh.n_omega && kh >= 0 && kh < sh.hist_cap)
                    ? sh.hist + ((size_t)kh * sh.n_omega + si) * 3 : nullptr;
    if (hrec) { hrec[0] = {0.0, 0.0}; hrec[1] = {0.0, 0.0}; hrec[2] = {0.0, 0.0}; }
    if (active) {
        const int k = s.k - 1;   // iteration just computed by the seed kernel
        dcx pc = sh.pi_cur[o], pp = sh.pi_prev[o], pt = sh.ptil[o], G = sh.G[o];
        const dcx alpha = {s.alpha_re, s.alpha_im}, c = {s.c_re, s.c_im};
        const dcx beta = {s.beta_prev_re, s.beta_prev_im}, g = {s.g_re, s.g_im};
        const dcx zs = sh.shift[s.seed_idx], zo = sh.shift[si];
        const dcx D = {zo.re - zs.re, zo.im - zs.im};
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
        if (hrec) { hrec[0] = as; hrec[1] = bs; hrec[2] = cdiv({1.0, 0.0}, pc); }
        const double f = s.rescale;   // range guard of the seed kernel (1 or a power of two)
        pc.re *= f; pc.im *= f; pn.re *= f; pn.im *= f;
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

// ------------------------------------------------------------ seed switch
// Applies the scalings of a seed switch decided by the seed kernel (see
// seed_one): r_k and w_k times s1, r_{k-1} times s0, and pi^s_k, pi^s_{k-1}
// of every shift of that right-hand side likewise. A right-hand side without
// a switch in this iteration returns at once (the usual case).
__device__ __forceinline__ dcl dcl_of(double re, double im) { return {dfl_from(re), dfl_from(im)}; }
__global__ void __launch_bounds__(256) cocg_switch_kernel(SwitchArgs sw) {
    if (*sw.all_done) return;
    const int j = blockIdx.y;
    const CocgSeed &s = sw.seed[j];
    if (!s.sw) return;
    const dcx s1 = {s.s1_re, s.s1_im}, s0 = {s.s0_re, s.s0_im};
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (uint64_t q = t0; q < (uint64_t)sw.n_omega; q += stride) {
        const size_t o = (size_t)j * sw.n_omega + q;
        sw.pi_cur[o] = cmul(sw.pi_cur[o], s1);
        sw.pi_prev[o] = cmul(sw.pi_prev[o], s0);
    }
    const size_t off = (size_t)j * sw.dim;
    if (sw.kind == 0) {
        double2 *rc = reinterpret_cast<double2 *>(sw.rcur) + off, *rp = reinterpret_cast<double2 *>(sw.rprev) + off;
        double2 *w = reinterpret_cast<double2 *>(sw.w) + off;
        for (uint64_t x = t0; x < sw.dim; x += stride) {
            const dcx a = cmul({rc[x].x, rc[x].y}, s1), b = cmul({rp[x].x, rp[x].y}, s0), c = cmul({w[x].x, w[x].y}, s1);
            rc[x] = make_double2(a.re, a.im); rp[x] = make_double2(b.re, b.im); w[x] = make_double2(c.re, c.im);
        }
    } else if (sw.kind == 1) {
        float2 *rc = reinterpret_cast<float2 *>(sw.rcur) + off, *rp = reinterpret_cast<float2 *>(sw.rprev) + off;
        float2 *w = reinterpret_cast<float2 *>(sw.w) + off;
        for (uint64_t x = t0; x < sw.dim; x += stride) {
            const dcx a = cmul({rc[x].x, rc[x].y}, s1), b = cmul({rp[x].x, rp[x].y}, s0), c = cmul({w[x].x, w[x].y}, s1);
            rc[x] = make_float2((float)a.re, (float)a.im); rp[x] = make_float2((float)b.re, (float)b.im);
            w[x] = make_float2((float)c.re, (float)c.im);
        }
    } else {
        // float hi + lo pairs: products in double-float arithmetic
        const long long lo = sw.lo_stride;
        float2 *rc = reinterpret_cast<float2 *>(sw.rcur) + off, *rp = reinterpret_cast<float2 *>(sw.rprev) + off;
        float2 *w = reinterpret_cast<float2 *>(sw.w) + off;
        const dcl f1 = dcl_of(s1.re, s1.im), f0 = dcl_of(s0.re, s0.im);
        for (uint64_t x = t0; x < sw.dim; x += stride) {
            const dcl a = dcl_mul({{rc[x].x, rc[x + lo].x}, {rc[x].y, rc[x + lo].y}}, f1);
            const dcl b = dcl_mul({{rp[x].x, rp[x + lo].x}, {rp[x].y, rp[x + lo].y}}, f0);
            rc[x] = make_float2(a.re.hi, a.im.hi); rc[x + lo] = make_float2(a.re.lo, a.im.lo);
            rp[x] = make_float2(b.re.hi, b.im.hi); rp[x + lo] = make_float2(b.re.lo, b.im.lo);
            if (sw.w_lo) {
                const dcl c = dcl_mul({{w[x].x, w[x + sw.w_lo].x}, {w[x].y, w[x + sw.w_lo].y}}, f1);
                w[x] = make_float2(c.re.hi, c.im.hi); w[x + sw.w_lo] = make_float2(c.re.lo, c.im.lo);
            } else {
                const dcx c = cmul({w[x].x, w[x].y}, s1);
                w[x] = make_float2((float)c.re, (float)c.im);
            }
        }
    }
}

// ------------------------------------------------------------ contour filter
// Second pass of the filter solve: phi_m += C[k][m] r_k for every centre m
// (FP64 vectors; k = iteration just computed, skipped once the solve is done).
__global__ void __launch_bounds__(256) filter_acc_kernel(FilterAccArgs fa) {
    const CocgSeed &s = *fa.seed;
    if (s.done) return;
    const int k = s.k - 1;
    if (k < 0 || k >= fa.n_coef) return;
    const dcx *c = fa.coef + (size_t)k * fa.L;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < fa.dim;
         x += (uint64_t)gridDim.x * blockDim.x) {
        const double2 r = fa.r[x];
        for (int m = 0; m < fa.L; ++m) {
            const dcx cm = c[m];
            double2 *p = fa.phi + (size_t)m * fa.dim + x;
            double2 v = *p;
            v.x = fma(cm.re, r.x, fma(-cm.im, r.y, v.x));
            v.y = fma(cm.re, r.y, fma(cm.im, r.x, v.y));
            *p = v;
        }
    }
}

// Filter coefficients: one CTA (one warp) per centre m, lane j < M the shift
// s = m M + j. Backward over the recorded iterations,
//   T^s_k = alpha^s_k + b^s_{k+1} T^s_{k+1}   (b^s_l = beta^s_{l-1}),
// so that x^s = sum_k (T^s_k / pi^s_k) r_k, and C[k][m] = sum_j w_j T^s_k / pi^s_k
// (warp sum in a fixed order).
__global__ void __launch_bounds__(32) filter_coef_kernel(FilterCoefArgs fc) {
    const int m = blockIdx.x, j = threadIdx.x;
    const bool on = j < fc.M;
    const size_t ns = (size_t)fc.L * fc.M;
    const size_t sidx = (size_t)m * fc.M + (on ? j : 0);
    const dcx wj = on ? fc.w[j] : dcx{0.0, 0.0};
    dcx T = {0.0, 0.0};
    for (int k = fc.n_iter - 1; k >= 0; --k) {
        dcx v = {0.0, 0.0};
        if (on) {
            const dcx *h = fc.hist + ((size_t)k * ns + sidx) * 3;
            const dcx bnext = (k + 1 < fc.n_iter) ? fc.hist[((size_t)(k + 1) * ns + sidx) * 3 + 1] : dcx{0.0, 0.0};
            const dcx bt = cmul(bnext, T);
            T = {h[0].re + bt.re, h[0].im + bt.im};
            v = cmul(wj, cmul(T, h[2]));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v.re += __shfl_xor_sync(0xffffffffu, v.re, o);
            v.im += __shfl_xor_sync(0xffffffffu, v.im, o);
        }
        if (j == 0) fc.coef[(size_t)k * fc.L + m] = v;
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

// ------------------------------------------------- filter-shell reweighting
__global__ void __launch_bounds__(256) frw_spectrum_kernel(FrwArgs fa) {
    __shared__ double red[(256 / 32) * 1];
    const int t = blockIdx.x;
    const double db = fa.beta - 1.0 / fa.T[t];
    double m = -INFINITY;
    for (int q = threadIdx.x; q < fa.n_shell; q += blockDim.x)
        if (fa.norm2[q] > 0.0) m = fmax(m, db * fa.E[q] + log(fa.norm2[q]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double mm = -INFINITY;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = fmax(mm, red[w]);
        double z = 0.0;   // fixed-order sum
        for (int q = 0; q < fa.n_shell; ++q)
            if (fa.norm2[q] > 0.0) z += exp(db * fa.E[q] + log(fa.norm2[q]) - mm);
        red[0] = mm;
        red[1] = z;
    }
    __syncthreads();
    const double mx = red[0], z = red[1];
    if (fa.P)
        for (int q = threadIdx.x; q < fa.n_shell; q += blockDim.x)
            fa.P[(size_t)t * fa.n_shell + q] =
                fa.norm2[q] > 0.0 ? exp(db * fa.E[q] + log(fa.norm2[q]) - mx) / (2.0 * fa.eps * z) : 0.0;
    for (int w = threadIdx.x; w < fa.n_omega; w += blockDim.x) {
        double acc = 0.0;
        // e^{db E_q} G_q = e^{db E_q + log n_q - mx} (G_q / n_q) e^{mx}: no
        // overflow for shells of tiny weight (G_q scales with n_q)
        for (int q = 0; q < fa.n_shell; ++q)
            if (fa.norm2[q] > 0.0)
                acc += exp(db * fa.E[q] + log(fa.norm2[q]) - mx) *
                       (-fa.G[2 * ((size_t)q * fa.n_omega + w) + 1] / M_PI / fa.norm2[q]);
        fa.S[(size_t)t * fa.n_omega + w] = acc / z;
    }
}

// ================================================================ launchers
cudaError_t launch_frw_spectrum(const FrwArgs &fa, int n_T, cudaStream_t st) {
    frw_spectrum_kernel<<<n_T, 256, 0, st>>>(fa);
    return cudaGetLastError();
}

cudaError_t launch_cocg_update(int kind, int B, void *rcur, const void *w, void *rprev_new,
                               const UpdArgs &ua, int grid, cudaStream_t st) {
    if (B < 1 || B > FTK_MAX_RHS) return cudaErrorInvalidValue;
    const dim3 g(grid, B);
    if (kind == 0) {
        PlainVec<double> v{reinterpret_cast<double2 *>(rcur), reinterpret_cast<const double2 *>(w),
                           reinterpret_cast<double2 *>(rprev_new)};
        cocg_update_kernel<<<g, 256, 0, st>>>(v, ua);
    } else if (kind == 1) {
        PlainVec<float> v{reinterpret_cast<float2 *>(rcur), reinterpret_cast<const float2 *>(w),
                          reinterpret_cast<float2 *>(rprev_new)};
        cocg_update_kernel<<<g, 256, 0, st>>>(v, ua);
    } else {
        cocg_update_df_kernel<<<g, 256, 0, st>>>(reinterpret_cast<float2 *>(rcur), reinterpret_cast<const float2 *>(w),
                                                reinterpret_cast<float2 *>(rprev_new), ua);
    }
    return cudaGetLastError();
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

cudaError_t launch_cocg_switch(const SwitchArgs &sw, int B, int grid, cudaStream_t st) {
    cocg_switch_kernel<<<dim3(grid, B), 256, 0, st>>>(sw);
    return cudaGetLastError();
}

cudaError_t launch_filter_acc(const FilterAccArgs &fa, int grid, cudaStream_t st) {
    filter_acc_kernel<<<grid, 256, 0, st>>>(fa);
    return cudaGetLastError();
}

cudaError_t launch_filter_coef(const FilterCoefArgs &fc, cudaStream_t st) {
    if (fc.M < 1 || fc.M > 32 || fc.L < 1) return cudaErrorInvalidValue;
    filter_coef_kernel<<<fc.L, 32, 0, st>>>(fc);
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
