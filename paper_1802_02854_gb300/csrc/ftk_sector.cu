// Momentum sectors of the translation group (the reduced-basis route to
// larger clusters; the paper itself works in the full basis, Sec. V).
//
// A group G of site permutations (the translations of the torus, N/2 of
// them) acts on basis states, g|x> = |g.x>, bit g(l) of g.x = bit l of x, and
// commutes with H. A sector is a one-dimensional character chi of G (chi(g) =
// e^{-i k.a_g} for the translation by a_g at momentum k); its projector is
//   P = (1/|G|) sum_g chi(g)^* g,   g P = chi(g) P.
// The orbit of a state has one representative r (the smallest integer in it);
// P|r> vanishes unless chi = 1 on the stabiliser of r, and then the sector
// basis vector is |r>_k = sqrt(o_r) P|r> with o_r the orbit size. With
// s = g.r' (r' the representative of s), P|s> = chi(g) P|r'>, so
//   <r'|H|r>_k = sum over the bonds b of r with rep(flip_b r) = r' of
//                c_b(r) chi(g_b) sqrt(o_r / o_r'),
// and since H_k is Hermitian the product is a gather over the bonds of the
// output representative:
//   (H v)_r' = D(r') v_r' + sum_b c_b(r') chi(g_b)^* sqrt(o_r' / o_r'') v_r'',
//   r'' = rep(flip_b r'), flip_b r' = g_b . r''.
// Data on the device: loc[x] = (orbit index << 5) | g for every state x
// (g . rep = x), the representatives and stabiliser masks of all orbits, and
// per sector the map orbit -> sector index (-1 where chi is not 1 on the
// stabiliser) and sqrt(o) per sector index. FP64 complex sector vectors.
//
// The sector Hamiltonian is complex Hermitian, not real symmetric, so the
// bilinear COCG of the full basis does not apply; the Green's function of a
// sector uses the Hermitian Lanczos process with the shifted recurrences of
// the LDL^T factors of z - T_j (one set of vectors for every shift):
//   d_0 = z - a_0,  d_j = z - a_j - b_j^2 / d_{j-1},  y_0 = 1,  y_j = y_{j-1} b_j / d_{j-1},
//   G_j(z) = |lambda|^2 sum_{i <= j} y_i^2 / d_i,
// and the shifted residual |r_j(z)| = |lambda| |b_{j+1} y_j / d_j| (the last
// component of the Galerkin solution times b_{j+1}), the criterion of the
// full-basis solve.
#include "../../include/ftk.h"
#include "ftk_common.cuh"
#include "ftk_device.cuh"
#include "ftk_kernels.h"
#include "ftk_plan.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <string>
#include <vector>

using namespace ftk;

namespace {

__device__ __forceinline__ dcx zmul(dcx a, dcx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ dcx zdiv(dcx a, dcx b) {   // Smith's algorithm
    if (fabs(b.re) >= fabs(b.im)) {
        const double r = b.im / b.re, d = b.re + b.im * r;
        return {(a.re + a.im * r) / d, (a.im - a.re * r) / d};
    }
    const double r = b.re / b.im, d = b.re * r + b.im;
    return {(a.re * r + a.im) / d, (a.im * r - a.re) / d};
}
__device__ __forceinline__ double zabs(dcx a) { return hypot(a.re, a.im); }

constexpr int kMaxGroup = 32;      // group elements (5 bits in loc)
constexpr int kSecThreads = 256;
constexpr int kScanBlock = 4096;   // states per counting block

struct SecGroup {
    int n, ng, nbytes;
    const uint32_t *tab;           // [ng][nbytes][256] bit images of the bytes of x
    int ginv[kMaxGroup];           // inverse element
};

__device__ __forceinline__ uint32_t act(const SecGroup &G, const uint32_t *tab, int g, uint32_t x) {
    uint32_t y = 0;
    for (int p = 0; p < G.nbytes; ++p) y |= tab[((size_t)g * G.nbytes + p) * 256 + ((x >> (8 * p)) & 255u)];
    return y;
}

// rep_of[x] = min_g g.x, g_of[x] = the element mapping the representative to x
// (the inverse of the smallest minimising element)
__global__ void __launch_bounds__(kSecThreads) sec_scan_kernel(SecGroup G, uint64_t dim, uint32_t *rep_of,
                                                               uint8_t *g_of) {
    extern __shared__ uint32_t stab[];
    const int nt = G.ng * G.nbytes * 256;
    for (int i = threadIdx.x; i < nt; i += blockDim.x) stab[i] = G.tab[i];
    __syncthreads();
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < dim; x += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t best = 0xffffffffu;
        int bg = 0;
        for (int g = 0; g < G.ng; ++g) {
            const uint32_t y = act(G, stab, g, (uint32_t)x);
            if (y < best) { best = y; bg = g; }
        }
        rep_of[x] = best;
        g_of[x] = (uint8_t)G.ginv[bg];
    }
}

// count of representatives per block of kScanBlock states
__global__ void __launch_bounds__(kSecThreads) sec_count_kernel(uint64_t dim, const uint32_t *rep_of, int *counts) {
    __shared__ int c;
    if (threadIdx.x == 0) c = 0;
    __syncthreads();
    const uint64_t b0 = (uint64_t)blockIdx.x * kScanBlock;
    int mine = 0;
    for (int i = threadIdx.x; i < kScanBlock; i += blockDim.x) {
        const uint64_t x = b0 + i;
        if (x < dim && rep_of[x] == (uint32_t)x) ++mine;
    }
    atomicAdd(&c, mine);   // integer: order-independent
    __syncthreads();
    if (threadIdx.x == 0) counts[blockIdx.x] = c;
}

// orbits in ascending order of their representative: orb_rep, stabiliser
// mask, and idx_of[rep] = orbit index
__global__ void __launch_bounds__(kSecThreads) sec_compact_kernel(SecGroup G, uint64_t dim, const uint32_t *rep_of,
                                                                  const int *offsets, uint32_t *orb_rep,
                                                                  uint32_t *orb_stab, int32_t *idx_of) {
    extern __shared__ uint32_t stab[];
    const int nt = G.ng * G.nbytes * 256;
    for (int i = threadIdx.x; i < nt; i += blockDim.x) stab[i] = G.tab[i];
    __shared__ int warp_tot[kSecThreads / 32];
    __shared__ int base;
    if (threadIdx.x == 0) base = offsets[blockIdx.x];
    __syncthreads();
    const uint64_t b0 = (uint64_t)blockIdx.x * kScanBlock;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c0 = 0; c0 < kScanBlock; c0 += blockDim.x) {
        const uint64_t x = b0 + c0 + threadIdx.x;
        const bool is_rep = x < dim && rep_of[x] == (uint32_t)x;
        const unsigned ball = __ballot_sync(0xffffffffu, is_rep);
        const int before = __popc(ball & ((1u << lane) - 1u));
        if (lane == 0) warp_tot[warp] = __popc(ball);
        __syncthreads();
        int wbase = 0;
        for (int w = 0; w < warp; ++w) wbase += warp_tot[w];
        if (is_rep) {
            const int o = base + wbase + before;
            uint32_t m = 0;
            for (int g = 0; g < G.ng; ++g)
                if (act(G, stab, g, (uint32_t)x) == (uint32_t)x) m |= 1u << g;
            orb_rep[o] = (uint32_t)x;
            orb_stab[o] = m;
            idx_of[x] = o;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += warp_tot[w];
            base += t;
        }
        __syncthreads();
    }
}

// loc[x] = orbit index * 32 + g (unsigned: up to 2^27 orbits)
__global__ void sec_loc_kernel(uint64_t dim, const uint32_t *rep_of, const uint8_t *g_of, const int32_t *idx_of,
                               uint32_t *loc) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < dim; x += (uint64_t)gridDim.x * blockDim.x)
        loc[x] = ((uint32_t)idx_of[rep_of[x]] << 5) | (uint32_t)g_of[x];
}

// sector basis: the orbits on whose stabiliser chi is 1 (flag, then compaction
// in orbit order); sqo = sqrt(|G| / |stabiliser|)
__global__ void sec_valid_kernel(int n_orb, int ng, const uint32_t *orb_stab, const double2 *chi, int *flag) {
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < n_orb; o += gridDim.x * blockDim.x) {
        const uint32_t m = orb_stab[o];
        int ok = 1;
        for (int g = 0; g < ng; ++g)
            if ((m >> g) & 1u) ok &= (fabs(chi[g].x - 1.0) < 1e-9 && fabs(chi[g].y) < 1e-9);
        flag[o] = ok;
    }
}

__global__ void sec_fill_kernel(int n_orb, int ng, const uint32_t *orb_stab, const int *flag, const int *pos,
                                int32_t *sec_index, int32_t *sec_orbit, double *sqo) {
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < n_orb; o += gridDim.x * blockDim.x) {
        if (!flag[o]) { sec_index[o] = -1; continue; }
        const int i = pos[o];
        sec_index[o] = i;
        sec_orbit[i] = o;
        sqo[i] = sqrt((double)ng / (double)__popc(orb_stab[o]));
    }
}

// ---------------------------------------------------------------- sector H.v
struct SecHam {
    int nb;
    uint32_t mask[2 * FTK_MAX_PASS_BONDS];
    uint8_t bi[2 * FTK_MAX_PASS_BONDS];
    double par[2 * FTK_MAX_PASS_BONDS], anti[2 * FTK_MAX_PASS_BONDS], dg[2 * FTK_MAX_PASS_BONDS];
};

enum { SEC_PLAIN = 0, SEC_TPQ = 1, SEC_DOT = 2 };

struct SecHvArgs {
    int64_t dim;
    const uint32_t *loc;
    const uint32_t *orb_rep;
    const int32_t *sec_index, *sec_orbit;
    const double *sqo;
    const double2 *chi;       // [ng]
    const double2 *in;
    double2 *out;
    double ell, inv_n;        // SEC_TPQ: out = ell v - H v / N
    const double *in_scale;   // optional device scale of the input (NULL: 1)
    double *partials;         // [grid][3]
    unsigned int *counter;
    double *result;           // [3]: <v|Hv>, |out|^2, |v|^2 (SEC_TPQ / SEC_DOT)
};

template <int EPI>
__global__ void __launch_bounds__(kSecThreads) sec_hv_kernel(const SecHam h, SecHvArgs a) {
    __shared__ double red[(kSecThreads / 32) * 3];
    const double sc = a.in_scale ? *a.in_scale : 1.0;
    double d0 = 0, d1 = 0, d2 = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.dim; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t r = a.orb_rep[a.sec_orbit[i]];
        const double so = a.sqo[i];
        const double2 v = a.in[i];
        double diag = 0, ar = 0, ai = 0;
        for (int b = 0; b < h.nb; ++b) {
            const uint32_t m = h.mask[b];
            const int par = (__popc(r & m) & 1) == 0;   // parallel spins
            diag += par ? h.dg[b] : -h.dg[b];
            const double c = par ? h.par[b] : h.anti[b];
            if (c == 0.0) continue;
            const uint32_t L = a.loc[r ^ m];
            const int32_t j = a.sec_index[L >> 5];
            if (j < 0) continue;
            const double2 ch = a.chi[L & 31];
            const double2 w = a.in[j];
            const double f = c * so / a.sqo[j];
            // conj(chi) w
            ar += f * (ch.x * w.x + ch.y * w.y);
            ai += f * (ch.x * w.y - ch.y * w.x);
        }
        ar = (ar + diag * v.x) * sc;
        ai = (ai + diag * v.y) * sc;
        if (EPI == SEC_PLAIN) {
            a.out[i] = make_double2(ar, ai);
        } else if (EPI == SEC_TPQ) {
            const double vx = v.x * sc, vy = v.y * sc;
            const double ox = a.ell * vx - a.inv_n * ar, oy = a.ell * vy - a.inv_n * ai;
            a.out[i] = make_double2(ox, oy);
            d0 += vx * ar + vy * ai;
            d1 += ox * ox + oy * oy;
            d2 += vx * vx + vy * vy;
        } else {
            a.out[i] = make_double2(ar, ai);
            const double vx = v.x * sc, vy = v.y * sc;
            d0 += vx * ar + vy * ai;
            d2 += vx * vx + vy * vy;
        }
    }
    if (EPI == SEC_PLAIN) return;
    double v3[3] = {d0, d1, d2};
    block_reduce<3>(v3, red);
    if (threadIdx.x < 3) a.partials[(size_t)blockIdx.x * 3 + threadIdx.x] = red[threadIdx.x];
    last_block_reduce<3>(a.partials, a.counter, a.result, red);
}

// --------------------------------------------------------- Lanczos vectors
// w = H q_j (in out, from SEC_DOT with a_j = <q_j|H q_j> in result[0]);
// w <- w - a_j q_j - b_j q_{j-1}, |w|^2 -> result; b_j from *beta_cur
struct LzArgs {
    int64_t dim;
    double2 *w;
    const double2 *q, *qp;
    const double *alpha;      // device a_j (the SEC_DOT result)
    const double *beta;       // device b_j (0 at j = 0)
    double *partials;
    unsigned int *counter;
    double *result;           // [1]: |w|^2
    const int *done;
};

__global__ void __launch_bounds__(kSecThreads) lz_update_kernel(LzArgs a) {
    __shared__ double red[kSecThreads / 32];
    if (*a.done) return;
    const double al = *a.alpha, be = *a.beta;
    double n2 = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.dim; i += (int64_t)gridDim.x * blockDim.x) {
        double2 w = a.w[i];
        const double2 q = a.q[i], p = a.qp[i];
        w.x = w.x - al * q.x - be * p.x;
        w.y = w.y - al * q.y - be * p.y;
        a.w[i] = w;
        n2 += w.x * w.x + w.y * w.y;
    }
    double v[1] = {n2};
    block_reduce<1>(v, red);
    if (threadIdx.x == 0) a.partials[blockIdx.x] = red[0];
    last_block_reduce<1>(a.partials, a.counter, a.result, red);
}

// q_{j+1} = w / b_{j+1} (in place of q_{j-1})
__global__ void lz_scale_kernel(int64_t dim, const double2 *w, double2 *qn, const double *beta_next, const int *done) {
    if (*done) return;
    const double b = *beta_next;
    const double s = b > 0 ? 1.0 / b : 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < dim; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 x = w[i];
        qn[i] = make_double2(x.x * s, x.y * s);
    }
}

// scalars of iteration j: a_j (alpha), b_{j+1} = sqrt(|w|^2); per shift the
// pivot d_j, y_j, G, frozen once |b_{j+1} y_j / d_j| <= tol; done when every
// shift is frozen, b_{j+1} vanished, or j + 1 = max_iter
struct LzShiftArgs {
    int n_shift, max_iter;
    double tol;
    const double2 *z;          // [n_shift]
    const double *alpha;       // a_j
    double *beta;              // [2]: b_j (read), b_{j+1} (written from w2)
    const double *w2;          // |w|^2
    double2 *d, *y, *G;        // [n_shift]
    int *frozen;               // [n_shift]
    int *iter;                 // j
    int *done;
    int *active_count;         // scratch: shifts still running after this iteration
};

__global__ void __launch_bounds__(256) lz_shift_kernel(LzShiftArgs a) {
    if (*a.done) return;
    const int j = *a.iter;
    const double al = *a.alpha, bj = a.beta[0];
    const double bn = sqrt(fmax(*a.w2, 0.0));
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    int mine = 0;
    for (int s = threadIdx.x; s < a.n_shift; s += blockDim.x) {
        if (a.frozen[s]) continue;
        const double2 z = a.z[s];
        dcx dn, yn;
        if (j == 0) {
            dn = {z.x - al, z.y};
            yn = {1.0, 0.0};
        } else {
            const double2 dp = a.d[s], yp = a.y[s];
            const dcx t = zdiv({bj * bj, 0.0}, {dp.x, dp.y});
            dn = {z.x - al - t.re, z.y - t.im};
            yn = zmul({yp.x, yp.y}, zdiv({bj, 0.0}, {dp.x, dp.y}));
        }
        const dcx term = zdiv(zmul(yn, yn), dn);
        double2 G = a.G[s];
        G.x += term.re;
        G.y += term.im;
        a.G[s] = G;
        a.d[s] = make_double2(dn.re, dn.im);
        a.y[s] = make_double2(yn.re, yn.im);
        const double res = bn * zabs(zdiv(yn, dn));
        if (res <= a.tol) a.frozen[s] = 1;
        else ++mine;
    }
    atomicAdd(&cnt, mine);
    __syncthreads();
    if (threadIdx.x == 0) {
        a.beta[0] = bn;   // b_{j+1} becomes b_j of the next iteration
        *a.iter = j + 1;
        if (cnt == 0 || bn == 0.0 || j + 1 >= a.max_iter) *a.done = (cnt == 0 || bn == 0.0) ? 1 : 2;
    }
}

// lambda_{k+q}[i] = f_q(r) psi_k[idx_k(r)] (S^z_q keeps the representative,
// f_q(r) = sum_l fq_l s_l(r), fq_l = N^{-1/2} e^{i q.R_l} / 2)
struct SzArgs {
    int64_t dim;               // destination sector
    int n;
    double2 fq[FTK_MAX_SITES];
    const uint32_t *orb_rep;
    const int32_t *dst_orbit, *src_index;
    const double2 *src;
    const double *src_scale;   // optional
    double2 *dst;
};

__global__ void sec_sz_kernel(SzArgs a) {
    const double sc = a.src_scale ? *a.src_scale : 1.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.dim; i += (int64_t)gridDim.x * blockDim.x) {
        const int o = a.dst_orbit[i];
        const int j = a.src_index[o];
        double2 out = make_double2(0.0, 0.0);
        if (j >= 0) {
            const uint32_t r = a.orb_rep[o];
            double fr = 0, fi = 0;
            for (int l = 0; l < a.n; ++l) {
                const double sg = ((r >> l) & 1u) ? 1.0 : -1.0;
                fr += sg * a.fq[l].x;
                fi += sg * a.fq[l].y;
            }
            const double2 p = a.src[j];
            out = make_double2(sc * (fr * p.x - fi * p.y), sc * (fr * p.y + fi * p.x));
        }
        a.dst[i] = out;
    }
}

// <r|_k psi = sqrt(o_r) <r|P|psi> = (sqrt(o_r)/|G|) sum_h chi(h)^* psi[h^{-1}.r]
struct ProjArgs {
    int64_t dim;
    SecGroup G;
    double2 chi[kMaxGroup];
    const uint32_t *orb_rep;
    const int32_t *sec_orbit;
    const double *sqo;
    const double2 *psi;        // full space
    double2 *out;
};

__global__ void __launch_bounds__(kSecThreads) sec_project_kernel(ProjArgs a) {
    extern __shared__ uint32_t stab[];
    const int nt = a.G.ng * a.G.nbytes * 256;
    for (int i = threadIdx.x; i < nt; i += blockDim.x) stab[i] = a.G.tab[i];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.dim; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t r = a.orb_rep[a.sec_orbit[i]];
        double sr = 0, si = 0;
        for (int h = 0; h < a.G.ng; ++h) {
            const double2 p = a.psi[act(a.G, stab, a.G.ginv[h], r)];
            const double2 c = a.chi[h];
            sr += c.x * p.x + c.y * p.y;   // conj(chi) psi
            si += c.x * p.y - c.y * p.x;
        }
        const double f = a.sqo[i] / a.G.ng;
        a.out[i] = make_double2(f * sr, f * si);
    }
}

__global__ void sec_scale_kernel(int64_t dim, const double2 *src, double2 *dst, const double *scale) {
    const double s = *scale;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < dim; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 x = src[i];
        dst[i] = make_double2(x.x * s, x.y * s);
    }
}

}  // namespace

// ---------------------------------------------------------------- objects
struct ftk_sector {
    ftk_ctx *ctx = nullptr;
    CtxHam ham{};
    int n = 0, ng = 0, nbytes = 0, n_orb = 0;
    uint64_t full_dim = 0;
    int64_t dim = 0;
    int n_slots = 0;
    std::vector<double> chi;             // [ng][2]
    std::vector<int> perm;               // [ng][n]
    std::vector<int> ginv;
    // device
    uint32_t *tab = nullptr;             // [ng][nbytes][256]
    uint32_t *loc = nullptr;             // [2^N]
    uint32_t *orb_rep = nullptr, *orb_stab = nullptr;   // [n_orb]
    int32_t *sec_index = nullptr;        // [n_orb]
    int32_t *sec_orbit = nullptr;        // [dim]
    double *sqo = nullptr;               // [dim]
    double2 *dchi = nullptr;             // [ng]
    double2 *vec = nullptr;              // [n_slots][dim]
    double *scal = nullptr;              // scalars / reductions: [0..63] results, then partials
    unsigned int *counter = nullptr;
    int *iflag = nullptr;                // [8]: done, iter, ...
    SecHam sh{};
    int grid = 0;
    bool owns_group = true;
};

namespace {

ftk_status sfail(ftk_sector *s, ftk_status st, const std::string &m) {
    if (s && s->ham.err) *s->ham.err = m;
    else set_thread_error(m.c_str());
    return st;
}

#define SCK(call)                                                                              \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) return sfail(sec, FTK_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)
#define SLAUNCH(call)                       \
    do {                                    \
        SCK(call);                          \
        ++*sec->ham.launches;               \
    } while (0)

constexpr int kPartialCap = 8192;   // reduction partials (grid cap)

double2 *slot_ptr(ftk_sector *s, int k) { return s->vec + (size_t)k * s->dim; }

int sec_grid(ftk_sector *s, int64_t n) {
    const int64_t want = (n + kSecThreads - 1) / kSecThreads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, std::min<int64_t>(kPartialCap, 8LL * s->ham.n_sm)));
}

SecGroup group_args(ftk_sector *s) {
    SecGroup g{};
    g.n = s->n;
    g.ng = s->ng;
    g.nbytes = s->nbytes;
    g.tab = s->tab;
    for (int i = 0; i < s->ng; ++i) g.ginv[i] = s->ginv[i];
    return g;
}

SecHvArgs hv_args(ftk_sector *s, const double2 *in, double2 *out) {
    SecHvArgs a{};
    a.dim = s->dim;
    a.loc = s->loc;
    a.orb_rep = s->orb_rep;
    a.sec_index = s->sec_index;
    a.sec_orbit = s->sec_orbit;
    a.sqo = s->sqo;
    a.chi = s->dchi;
    a.in = in;
    a.out = out;
    a.inv_n = 1.0 / s->n;
    a.partials = s->scal + 64;
    a.counter = s->counter;
    a.result = s->scal;
    return a;
}

}  // namespace

extern "C" {

ftk_status ftk_sector_create(ftk_ctx *ctx, const int32_t *perms, int32_t n_g, const double *chi, int32_t n_slots,
                             ftk_sector **out, int64_t *dim_out) {
    if (!out) return FTK_EINVAL;
    *out = nullptr;
    CtxHam h{};
    if (!ctx_hamiltonian(ctx, &h)) return FTK_EINVAL;
    ftk_sector *sec = nullptr;
    auto bad = [&](const char *m) { *h.err = m; return FTK_EINVAL; };
    if (!perms || !chi || n_g < 1 || n_g > kMaxGroup || n_slots < 1 || n_slots > 64)
        return bad("ftk_sector_create: bad arguments (1 <= n_g <= 32, 1 <= n_slots <= 64)");
    const int n = h.n;
    if (n > 30) return bad("ftk_sector_create: at most 30 sites");
    // the permutations must form a group (closure), start with the identity,
    // commute with H (map the bond list to itself, types kept), and chi must
    // be a unitary character of it
    std::vector<int> P(perms, perms + (size_t)n_g * n);
    for (int g = 0; g < n_g; ++g) {
        std::vector<int> seen(n, 0);
        for (int l = 0; l < n; ++l) {
            const int t = P[(size_t)g * n + l];
            if (t < 0 || t >= n || seen[t]) return bad("ftk_sector_create: a group element is not a permutation");
            seen[t] = 1;
        }
    }
    for (int l = 0; l < n; ++l)
        if (P[l] != l) return bad("ftk_sector_create: element 0 must be the identity");
    auto find = [&](const std::vector<int> &q) -> int {
        for (int g = 0; g < n_g; ++g)
            if (std::equal(q.begin(), q.end(), P.begin() + (size_t)g * n)) return g;
        return -1;
    };
    std::vector<int> mul((size_t)n_g * n_g);
    for (int a = 0; a < n_g; ++a)
        for (int b = 0; b < n_g; ++b) {
            std::vector<int> q(n);
            for (int l = 0; l < n; ++l) q[l] = P[(size_t)a * n + P[(size_t)b * n + l]];   // a after b
            const int c = find(q);
            if (c < 0) return bad("ftk_sector_create: the permutations are not closed under composition");
            mul[(size_t)a * n_g + b] = c;
        }
    for (int g = 0; g < n_g; ++g) {
        for (int q = 0; q < h.nb; ++q) {
            const int i = P[(size_t)g * n + h.bonds[3 * q]], j = P[(size_t)g * n + h.bonds[3 * q + 1]];
            bool ok = false;
            for (int r = 0; r < h.nb && !ok; ++r)
                ok = h.bonds[3 * r + 2] == h.bonds[3 * q + 2] &&
                     ((h.bonds[3 * r] == i && h.bonds[3 * r + 1] == j) || (h.bonds[3 * r] == j && h.bonds[3 * r + 1] == i));
            if (!ok) return bad("ftk_sector_create: a group element does not map the bond list to itself");
        }
    }
    for (int a = 0; a < n_g; ++a) {
        const std::complex<double> ca(chi[2 * a], chi[2 * a + 1]);
        if (std::abs(std::abs(ca) - 1.0) > 1e-9) return bad("ftk_sector_create: chi must have unit modulus");
        for (int b = 0; b < n_g; ++b) {
            const int c = mul[(size_t)a * n_g + b];
            const std::complex<double> cb(chi[2 * b], chi[2 * b + 1]), cc(chi[2 * c], chi[2 * c + 1]);
            if (std::abs(ca * cb - cc) > 1e-9) return bad("ftk_sector_create: chi is not a character of the group");
        }
    }
    sec = new (std::nothrow) ftk_sector();
    if (!sec) return FTK_ENOMEM;
    sec->ctx = ctx;
    sec->ham = h;
    sec->n = n;
    sec->ng = n_g;
    sec->nbytes = (n + 7) / 8;
    sec->full_dim = uint64_t(1) << n;
    sec->n_slots = n_slots;
    sec->chi.assign(chi, chi + 2 * n_g);
    sec->perm = P;
    sec->ginv.assign(n_g, 0);
    for (int a = 0; a < n_g; ++a)
        for (int b = 0; b < n_g; ++b)
            if (mul[(size_t)a * n_g + b] == 0) sec->ginv[a] = b;
    // bonds
    sec->sh.nb = h.nb;
    for (int q = 0; q < h.nb; ++q) {
        const int i = h.bonds[3 * q], j = h.bonds[3 * q + 1], g = h.bonds[3 * q + 2];
        sec->sh.mask[q] = (1u << i) | (1u << j);
        double pa = 0, an = 0;
        bond_coefficients(g, h.K, h.J, &pa, &an);
        sec->sh.par[q] = pa;
        sec->sh.anti[q] = an;
        sec->sh.dg[q] = g == 2 ? (h.J + h.K) / 4 : h.J / 4;
    }
    // byte tables: image of byte value v at byte position p under g
    std::vector<uint32_t> tab((size_t)n_g * sec->nbytes * 256, 0);
    for (int g = 0; g < n_g; ++g)
        for (int p = 0; p < sec->nbytes; ++p)
            for (int v = 0; v < 256; ++v) {
                uint32_t y = 0;
                for (int b = 0; b < 8; ++b) {
                    const int l = 8 * p + b;
                    if (l < n && ((v >> b) & 1)) y |= 1u << P[(size_t)g * n + l];
                }
                tab[((size_t)g * sec->nbytes + p) * 256 + v] = y;
            }
    cudaStream_t st = h.stream;
    const uint64_t D = sec->full_dim;
    const int n_blocks = (int)((D + kScanBlock - 1) / kScanBlock);
    uint32_t *rep_of = nullptr;
    uint8_t *g_of = nullptr;
    int32_t *idx_of = nullptr;
    int *counts = nullptr, *flag = nullptr, *fpos = nullptr;
    auto cleanup = [&]() {
        cudaFree(rep_of); cudaFree(g_of); cudaFree(idx_of); cudaFree(counts); cudaFree(flag); cudaFree(fpos);
    };
    auto fail_all = [&](ftk_status s_, const std::string &m) {
        cleanup();
        ftk_sector_destroy(sec);
        *h.err = m;
        return s_;
    };
#define CK2(call)                                                                                         \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess) return fail_all(FTK_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)
    const size_t tab_bytes = tab.size() * 4;
    // byte tables in shared memory: up to 32 elements x 4 bytes x 1 KB
    CK2(cudaFuncSetAttribute(sec_scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 << 10));
    CK2(cudaFuncSetAttribute(sec_compact_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 << 10));
    CK2(cudaFuncSetAttribute(sec_project_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 << 10));
    CK2(cudaMalloc(&sec->tab, tab_bytes));
    CK2(cudaMemcpyAsync(sec->tab, tab.data(), tab_bytes, cudaMemcpyHostToDevice, st));
    CK2(cudaMalloc(&sec->loc, D * 4));
    CK2(cudaMalloc(&rep_of, D * 4));
    CK2(cudaMalloc(&g_of, D));
    CK2(cudaMalloc(&idx_of, D * 4));
    CK2(cudaMalloc(&counts, sizeof(int) * n_blocks));
    SecGroup G = group_args(sec);
    const int ggrid = (int)std::min<uint64_t>((D + kSecThreads - 1) / kSecThreads, 16ull * h.n_sm);
    sec_scan_kernel<<<ggrid, kSecThreads, tab_bytes, st>>>(G, D, rep_of, g_of);
    CK2(cudaGetLastError());
    sec_count_kernel<<<n_blocks, kSecThreads, 0, st>>>(D, rep_of, counts);
    CK2(cudaGetLastError());
    std::vector<int> cnt(n_blocks), off(n_blocks);
    CK2(cudaMemcpyAsync(cnt.data(), counts, sizeof(int) * n_blocks, cudaMemcpyDeviceToHost, st));
    CK2(cudaStreamSynchronize(st));
    long tot = 0;
    for (int b = 0; b < n_blocks; ++b) { off[b] = (int)tot; tot += cnt[b]; }
    sec->n_orb = (int)tot;
    CK2(cudaMemcpyAsync(counts, off.data(), sizeof(int) * n_blocks, cudaMemcpyHostToDevice, st));
    CK2(cudaMalloc(&sec->orb_rep, 4 * (size_t)tot));
    CK2(cudaMalloc(&sec->orb_stab, 4 * (size_t)tot));
    sec_compact_kernel<<<n_blocks, kSecThreads, tab_bytes, st>>>(G, D, rep_of, counts, sec->orb_rep, sec->orb_stab, idx_of);
    CK2(cudaGetLastError());
    sec_loc_kernel<<<ggrid, kSecThreads, 0, st>>>(D, rep_of, g_of, idx_of, sec->loc);
    CK2(cudaGetLastError());
    // sector basis
    CK2(cudaMalloc(&sec->dchi, sizeof(double2) * n_g));
    CK2(cudaMemcpyAsync(sec->dchi, chi, sizeof(double2) * n_g, cudaMemcpyHostToDevice, st));
    CK2(cudaMalloc(&flag, sizeof(int) * tot));
    CK2(cudaMalloc(&fpos, sizeof(int) * tot));
    sec_valid_kernel<<<sec_grid(sec, tot), kSecThreads, 0, st>>>((int)tot, n_g, sec->orb_stab, sec->dchi, flag);
    CK2(cudaGetLastError());
    std::vector<int> fl(tot), pos(tot);
    CK2(cudaMemcpyAsync(fl.data(), flag, sizeof(int) * tot, cudaMemcpyDeviceToHost, st));
    CK2(cudaStreamSynchronize(st));
    int64_t dim = 0;
    for (long o = 0; o < tot; ++o) { pos[o] = (int)dim; dim += fl[o]; }
    sec->dim = dim;
    if (dim == 0) return fail_all(FTK_EINVAL, "ftk_sector_create: the sector is empty");
    CK2(cudaMemcpyAsync(fpos, pos.data(), sizeof(int) * tot, cudaMemcpyHostToDevice, st));
    CK2(cudaMalloc(&sec->sec_index, sizeof(int32_t) * tot));
    CK2(cudaMalloc(&sec->sec_orbit, sizeof(int32_t) * dim));
    CK2(cudaMalloc(&sec->sqo, sizeof(double) * dim));
    sec_fill_kernel<<<sec_grid(sec, tot), kSecThreads, 0, st>>>((int)tot, n_g, sec->orb_stab, flag, fpos, sec->sec_index,
                                                                 sec->sec_orbit, sec->sqo);
    CK2(cudaGetLastError());
    CK2(cudaMalloc(&sec->vec, sizeof(double2) * (size_t)dim * n_slots));
    CK2(cudaMemsetAsync(sec->vec, 0, sizeof(double2) * (size_t)dim * n_slots, st));
    CK2(cudaMalloc(&sec->scal, sizeof(double) * (64 + 3 * kPartialCap)));
    CK2(cudaMemsetAsync(sec->scal, 0, sizeof(double) * 64, st));
    CK2(cudaMalloc(&sec->counter, sizeof(unsigned int) * 4));
    CK2(cudaMemsetAsync(sec->counter, 0, sizeof(unsigned int) * 4, st));
    CK2(cudaMalloc(&sec->iflag, sizeof(int) * 8));
    CK2(cudaMemsetAsync(sec->iflag, 0, sizeof(int) * 8, st));
    CK2(cudaStreamSynchronize(st));
#undef CK2
    cleanup();
    *h.launches += 7;
    *out = sec;
    if (dim_out) *dim_out = dim;
    return FTK_OK;
}

void ftk_sector_destroy(ftk_sector *s) {
    if (!s) return;
    if (s->ham.stream) cudaStreamSynchronize(s->ham.stream);
    cudaFree(s->tab); cudaFree(s->loc); cudaFree(s->orb_rep); cudaFree(s->orb_stab); cudaFree(s->sec_index);
    cudaFree(s->sec_orbit); cudaFree(s->sqo); cudaFree(s->dchi); cudaFree(s->vec); cudaFree(s->scal);
    cudaFree(s->counter); cudaFree(s->iflag);
    delete s;
}

ftk_status ftk_sector_info(const ftk_sector *s, int64_t *dim, int32_t *n_orbits, uint32_t *reps_host) {
    ftk_sector *sec = const_cast<ftk_sector *>(s);
    if (!sec) return FTK_EINVAL;
    if (dim) *dim = sec->dim;
    if (n_orbits) *n_orbits = sec->n_orb;
    if (reps_host) {
        std::vector<int32_t> orb(sec->dim);
        std::vector<uint32_t> rep(sec->n_orb);
        SCK(cudaMemcpyAsync(orb.data(), sec->sec_orbit, sizeof(int32_t) * sec->dim, cudaMemcpyDeviceToHost, sec->ham.stream));
        SCK(cudaMemcpyAsync(rep.data(), sec->orb_rep, sizeof(uint32_t) * sec->n_orb, cudaMemcpyDeviceToHost, sec->ham.stream));
        SCK(cudaStreamSynchronize(sec->ham.stream));
        for (int64_t i = 0; i < sec->dim; ++i) reps_host[i] = rep[orb[i]];
    }
    return FTK_OK;
}

ftk_status ftk_sector_set(ftk_sector *sec, int32_t slot, const double *v, int32_t is_device) {
    if (!sec || !v || slot < 0 || slot >= sec->n_slots) return sfail(sec, FTK_EINVAL, "ftk_sector_set: bad arguments");
    SCK(cudaMemcpyAsync(slot_ptr(sec, slot), v, sizeof(double2) * sec->dim,
                        is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, sec->ham.stream));
    SCK(cudaStreamSynchronize(sec->ham.stream));
    return FTK_OK;
}

ftk_status ftk_sector_get(ftk_sector *sec, int32_t slot, double *host_out) {
    if (!sec || !host_out || slot < 0 || slot >= sec->n_slots) return sfail(sec, FTK_EINVAL, "ftk_sector_get: bad arguments");
    SCK(cudaMemcpyAsync(host_out, slot_ptr(sec, slot), sizeof(double2) * sec->dim, cudaMemcpyDeviceToHost, sec->ham.stream));
    SCK(cudaStreamSynchronize(sec->ham.stream));
    return FTK_OK;
}

ftk_status ftk_sector_project(ftk_sector *sec, const double *psi_full, int32_t is_device, int32_t slot) {
    if (!sec || !psi_full || slot < 0 || slot >= sec->n_slots) return sfail(sec, FTK_EINVAL, "ftk_sector_project: bad arguments");
    const double2 *src = reinterpret_cast<const double2 *>(psi_full);
    double2 *stage = nullptr;
    if (!is_device) {
        SCK(cudaMalloc(&stage, sizeof(double2) * sec->full_dim));
        SCK(cudaMemcpyAsync(stage, psi_full, sizeof(double2) * sec->full_dim, cudaMemcpyHostToDevice, sec->ham.stream));
        src = stage;
    }
    ProjArgs a{};
    a.dim = sec->dim;
    a.G = group_args(sec);
    for (int g = 0; g < sec->ng; ++g) a.chi[g] = make_double2(sec->chi[2 * g], sec->chi[2 * g + 1]);
    a.orb_rep = sec->orb_rep;
    a.sec_orbit = sec->sec_orbit;
    a.sqo = sec->sqo;
    a.psi = src;
    a.out = slot_ptr(sec, slot);
    const size_t tab_bytes = (size_t)sec->ng * sec->nbytes * 256 * 4;
    sec_project_kernel<<<sec_grid(sec, sec->dim), kSecThreads, tab_bytes, sec->ham.stream>>>(a);
    cudaError_t e = cudaGetLastError();
    ++*sec->ham.launches;
    if (e == cudaSuccess) e = cudaStreamSynchronize(sec->ham.stream);
    if (stage) cudaFree(stage);
    if (e != cudaSuccess) return sfail(sec, FTK_ECUDA, cudaGetErrorString(e));
    return FTK_OK;
}

ftk_status ftk_sector_hv(ftk_sector *sec, int32_t slot_in, int32_t slot_out) {
    if (!sec || slot_in < 0 || slot_out < 0 || slot_in >= sec->n_slots || slot_out >= sec->n_slots || slot_in == slot_out)
        return sfail(sec, FTK_EINVAL, "ftk_sector_hv: bad slots");
    SecHvArgs a = hv_args(sec, slot_ptr(sec, slot_in), slot_ptr(sec, slot_out));
    sec_hv_kernel<SEC_PLAIN><<<sec_grid(sec, sec->dim), kSecThreads, 0, sec->ham.stream>>>(sec->sh, a);
    SCK(cudaGetLastError());
    ++*sec->ham.launches;
    return FTK_OK;
}

ftk_status ftk_sector_tpq(ftk_sector *sec, int32_t slot_state, int32_t slot_work, double ell, int32_t n_steps,
                          int32_t save_every, int32_t first_save_slot, double *u_out, double *logq_out,
                          double *lognorm0_out) {
    if (!sec || slot_state < 0 || slot_work < 0 || slot_state >= sec->n_slots || slot_work >= sec->n_slots ||
        slot_state == slot_work || n_steps < 0 || save_every < 1 || first_save_slot < 0)
        return sfail(sec, FTK_EINVAL, "ftk_sector_tpq: bad arguments");
    if (!(ell >= sec->ham.ell_min - 1e-12)) return sfail(sec, FTK_EINVAL, "ftk_sector_tpq: ell below l_min");
    int n_save = 0;
    for (int k = 0; k < n_steps; ++k) n_save += (k % save_every == 0);
    if (n_save > 0 && first_save_slot + n_save > sec->n_slots)
        return sfail(sec, FTK_EINVAL, "ftk_sector_tpq: not enough slots for the saved states");
    for (int k = 0; k < n_save; ++k)
        if (first_save_slot + k == slot_state || first_save_slot + k == slot_work)
            return sfail(sec, FTK_EINVAL, "ftk_sector_tpq: save slots overlap the state or work slot");
    cudaStream_t st = sec->ham.stream;
    // normalise the initial state (its norm is returned: the sector's share of
    // a projected state)
    {
        SecHvArgs a = hv_args(sec, slot_ptr(sec, slot_state), slot_ptr(sec, slot_work));
        sec_hv_kernel<SEC_DOT><<<sec_grid(sec, sec->dim), kSecThreads, 0, st>>>(sec->sh, a);
        SCK(cudaGetLastError());
        ++*sec->ham.launches;
        double r[3];
        SCK(cudaMemcpyAsync(r, sec->scal, sizeof r, cudaMemcpyDeviceToHost, st));
        SCK(cudaStreamSynchronize(st));
        if (!(r[2] > 0)) return sfail(sec, FTK_EINVAL, "ftk_sector_tpq: the state has no component in this sector");
        if (lognorm0_out) *lognorm0_out = 0.5 * std::log(r[2]);
        const double sc = 1.0 / std::sqrt(r[2]);
        SCK(cudaMemcpyAsync(sec->scal + 8, &sc, sizeof sc, cudaMemcpyHostToDevice, st));
        sec_scale_kernel<<<sec_grid(sec, sec->dim), kSecThreads, 0, st>>>(sec->dim, slot_ptr(sec, slot_state),
                                                                           slot_ptr(sec, slot_state), sec->scal + 8);
        SCK(cudaGetLastError());
        ++*sec->ham.launches;
    }
    double logq = 0.0;
    int saved = 0;
    for (int k = 0; k < n_steps; ++k) {
        double2 *cur = slot_ptr(sec, slot_state), *wk = slot_ptr(sec, slot_work);
        if (k % save_every == 0) {
            SCK(cudaMemcpyAsync(slot_ptr(sec, first_save_slot + saved), cur, sizeof(double2) * sec->dim,
                                cudaMemcpyDeviceToDevice, st));
            ++saved;
        }
        SecHvArgs a = hv_args(sec, cur, wk);
        a.ell = ell;
        sec_hv_kernel<SEC_TPQ><<<sec_grid(sec, sec->dim), kSecThreads, 0, st>>>(sec->sh, a);
        SCK(cudaGetLastError());
        ++*sec->ham.launches;
        double r[3];
        SCK(cudaMemcpyAsync(r, sec->scal, sizeof r, cudaMemcpyDeviceToHost, st));
        SCK(cudaStreamSynchronize(st));
        // u_k = <psi_k|H|psi_k> / N (psi_k normalised); log Q_k; q_k = |psi'|
        if (u_out) u_out[k] = r[0] / sec->n;
        if (logq_out) logq_out[k] = logq;
        if (!(r[1] > 0)) return sfail(sec, FTK_EBREAKDOWN, "ftk_sector_tpq: the state vanished");
        logq += 0.5 * std::log(r[1]);
        const double sc = 1.0 / std::sqrt(r[1]);
        SCK(cudaMemcpyAsync(sec->scal + 8, &sc, sizeof sc, cudaMemcpyHostToDevice, st));
        sec_scale_kernel<<<sec_grid(sec, sec->dim), kSecThreads, 0, st>>>(sec->dim, wk, cur, sec->scal + 8);
        SCK(cudaGetLastError());
        ++*sec->ham.launches;
    }
    SCK(cudaStreamSynchronize(st));
    return FTK_OK;
}

ftk_status ftk_sector_apply_sz(ftk_sector *src, int32_t slot_src, ftk_sector *dst, int32_t slot_dst, const double q[2]) {
    ftk_sector *sec = dst;
    if (!src || !dst || !q || slot_src < 0 || slot_src >= src->n_slots || slot_dst < 0 || slot_dst >= dst->n_slots)
        return sfail(sec, FTK_EINVAL, "ftk_sector_apply_sz: bad arguments");
    if (src->ctx != dst->ctx || src->ng != dst->ng || src->perm != dst->perm || (src == dst && slot_src == slot_dst))
        return sfail(sec, FTK_EINVAL, "ftk_sector_apply_sz: the sectors must share the context and the group");
    // chi_dst(g) = chi_src(g) e^{-i q.a_g}, a_g = R_{g(0)} - R_0 (a cluster momentum q
    // makes the phase independent of the site used)
    const double *R = src->ham.pos;
    for (int g = 0; g < src->ng; ++g) {
        const int l = src->perm[(size_t)g * src->n];
        const double ph = -(q[0] * (R[2 * l] - R[0]) + q[1] * (R[2 * l + 1] - R[1]));
        const std::complex<double> want = std::complex<double>(src->chi[2 * g], src->chi[2 * g + 1]) *
                                          std::complex<double>(std::cos(ph), std::sin(ph));
        if (std::abs(want - std::complex<double>(dst->chi[2 * g], dst->chi[2 * g + 1])) > 1e-8)
            return sfail(sec, FTK_EINVAL, "ftk_sector_apply_sz: the destination sector is not the source's k + q");
    }
    SzArgs a{};
    a.dim = dst->dim;
    a.n = dst->n;
    const double nrm = 1.0 / std::sqrt((double)dst->n);
    for (int l = 0; l < dst->n; ++l) {
        const double ph = q[0] * R[2 * l] + q[1] * R[2 * l + 1];
        a.fq[l] = make_double2(0.5 * nrm * std::cos(ph), 0.5 * nrm * std::sin(ph));
    }
    a.orb_rep = dst->orb_rep;
    a.dst_orbit = dst->sec_orbit;
    a.src_index = src->sec_index;
    a.src = slot_ptr(src, slot_src);
    a.dst = slot_ptr(dst, slot_dst);
    sec_sz_kernel<<<sec_grid(dst, dst->dim), kSecThreads, 0, dst->ham.stream>>>(a);
    SCK(cudaGetLastError());
    ++*sec->ham.launches;
    SCK(cudaStreamSynchronize(dst->ham.stream));
    return FTK_OK;
}

ftk_status ftk_sector_green(ftk_sector *sec, int32_t slot, const double *shifts, int32_t n_shift, double tol,
                            int32_t max_iter, double *G_out, int32_t *iters_out) {
    if (!sec || slot < 0 || slot >= sec->n_slots || sec->n_slots < 4 || !shifts || n_shift < 1 ||
        n_shift > FTK_MAX_OMEGA || !(tol > 0) || max_iter < 1 || !G_out)
        return sfail(sec, FTK_EINVAL, "ftk_sector_green: bad arguments (needs 4 slots besides none: q, q', w use the "
                                      "three slots after the probe, cyclically)");
    cudaStream_t st = sec->ham.stream;
    // vectors: q_prev, q, w in the three slots after `slot` (cyclic)
    const int s1 = (slot + 1) % sec->n_slots, s2 = (slot + 2) % sec->n_slots, s3 = (slot + 3) % sec->n_slots;
    double2 *lam = slot_ptr(sec, slot), *qa = slot_ptr(sec, s1), *qb = slot_ptr(sec, s2), *w = slot_ptr(sec, s3);
    // |lambda|^2 and q_0 = lambda / |lambda|, q_{-1} = 0
    SecHvArgs a0 = hv_args(sec, lam, w);
    sec_hv_kernel<SEC_DOT><<<sec_grid(sec, sec->dim), kSecThreads, 0, st>>>(sec->sh, a0);
    SCK(cudaGetLastError());
    double r[3];
    SCK(cudaMemcpyAsync(r, sec->scal, sizeof r, cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    const double lam2 = r[2];
    if (!(lam2 > 0)) {   // a zero probe: G = 0
        std::fill(G_out, G_out + 2 * (size_t)n_shift, 0.0);
        if (iters_out) *iters_out = 0;
        return FTK_OK;
    }
    const double sc = 1.0 / std::sqrt(lam2);
    // device scalars (scal): [0..2] dot results, [8] scale, [16] alpha, [17..18] beta, [20] |w|^2
    SCK(cudaMemcpyAsync(sec->scal + 8, &sc, sizeof sc, cudaMemcpyHostToDevice, st));
    sec_scale_kernel<<<sec_grid(sec, sec->dim), kSecThreads, 0, st>>>(sec->dim, lam, qb, sec->scal + 8);
    SCK(cudaGetLastError());
    SCK(cudaMemsetAsync(qa, 0, sizeof(double2) * sec->dim, st));
    SCK(cudaMemsetAsync(sec->scal + 17, 0, sizeof(double) * 2, st));
    SCK(cudaMemsetAsync(sec->iflag, 0, sizeof(int) * 8, st));
    // per-shift state in a scratch allocation: z, d, y, G, frozen
    double2 *zd = nullptr;
    SCK(cudaMalloc(&zd, sizeof(double2) * 4 * n_shift + sizeof(int) * n_shift));
    double2 *dz = zd, *dd = zd + n_shift, *dy = zd + 2 * n_shift, *dG = zd + 3 * n_shift;
    int *dfz = reinterpret_cast<int *>(zd + 4 * n_shift);
    cudaError_t e = cudaMemcpyAsync(dz, shifts, sizeof(double2) * n_shift, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dd, 0, sizeof(double2) * 3 * n_shift + sizeof(int) * n_shift, st);
    if (e != cudaSuccess) { cudaFree(zd); return sfail(sec, FTK_ECUDA, cudaGetErrorString(e)); }
    LzShiftArgs la{};
    la.n_shift = n_shift;
    la.max_iter = max_iter;
    la.tol = tol;
    la.z = dz;
    la.alpha = sec->scal;          // SEC_DOT result[0] = <q|Hq> (q normalised, real part)
    la.beta = sec->scal + 17;
    la.w2 = sec->scal + 20;
    la.d = dd;
    la.y = dy;
    la.G = dG;
    la.frozen = dfz;
    la.iter = sec->iflag + 1;
    la.done = sec->iflag;
    int done = 0, it = 0;
    double2 *qp = qa, *qc = qb;    // q_{j-1}, q_j
    while (e == cudaSuccess) {
        for (int c = 0; c < 32 && it < max_iter; ++c, ++it) {
            // w = H q_j, a_j = <q_j|H q_j>; skipped once done (the dot kernel
            // itself runs, its result is unused)
            SecHvArgs a = hv_args(sec, qc, w);
            sec_hv_kernel<SEC_DOT><<<sec_grid(sec, sec->dim), kSecThreads, 0, st>>>(sec->sh, a);
            LzArgs u{};
            u.dim = sec->dim;
            u.w = w;
            u.q = qc;
            u.qp = qp;
            u.alpha = sec->scal;
            u.beta = sec->scal + 17;
            u.partials = sec->scal + 64;
            u.counter = sec->counter + 1;
            u.result = sec->scal + 20;
            u.done = sec->iflag;
            lz_update_kernel<<<sec_grid(sec, sec->dim), kSecThreads, 0, st>>>(u);
            lz_shift_kernel<<<1, 256, 0, st>>>(la);
            // q_{j+1} = w / b_{j+1} into q_{j-1}'s buffer
            lz_scale_kernel<<<sec_grid(sec, sec->dim), kSecThreads, 0, st>>>(sec->dim, w, qp, sec->scal + 17, sec->iflag);
            e = cudaGetLastError();
            if (e != cudaSuccess) break;
            *sec->ham.launches += 4;
            std::swap(qp, qc);
        }
        if (e != cudaSuccess) break;
        e = cudaMemcpyAsync(&done, sec->iflag, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (done || it >= max_iter) break;
    }
    std::vector<double> G(2 * (size_t)n_shift);
    int iters = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(G.data(), dG, sizeof(double2) * n_shift, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&iters, sec->iflag + 1, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&done, sec->iflag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(zd);
    if (e != cudaSuccess) return sfail(sec, FTK_ECUDA, cudaGetErrorString(e));
    for (size_t i = 0; i < G.size(); ++i) G_out[i] = lam2 * G[i];
    if (iters_out) *iters_out = iters;
    if (done != 1) return sfail(sec, FTK_ENOCONV, "ftk_sector_green: max_iter reached");
    return FTK_OK;
}

ftk_status ftk_sector_combine(int32_t n_sec, int32_t n_steps, const double *lognorm0, const double *logq,
                               const double *u, int32_t n_shell, const int32_t *shell_steps, int32_t n_omega,
                               const double *G, double *u_out, double *logQ_out, double *G_out) {
    // The full state is the direct sum of its sector parts: |(l - h)^k psi_0|^2
    // = sum_s e^{2 (lognorm0_s + logq_s[k])}; energies and Green's functions of
    // the normalised full state are the averages of the sectors' with the
    // weights e^{2 (lognorm0_s + logq_s[k])} (log-sum-exp)
    if (n_sec < 1 || n_steps < 1 || !lognorm0 || !logq || !u || !u_out || !logQ_out || n_shell < 0 ||
        (n_shell > 0 && (!shell_steps || !G || !G_out || n_omega < 1))) {
        set_thread_error("ftk_sector_combine: bad arguments");
        return FTK_EINVAL;
    }
    auto lse2 = [&](int k, std::vector<double> &w) {   // log sum e^{2 a_s}, weights e^{2 a_s - m}
        double m = -INFINITY;
        for (int s = 0; s < n_sec; ++s) m = std::max(m, 2.0 * (lognorm0[s] + logq[(size_t)s * n_steps + k]));
        double t = 0;
        w.assign(n_sec, 0.0);
        for (int s = 0; s < n_sec; ++s) {
            w[s] = std::exp(2.0 * (lognorm0[s] + logq[(size_t)s * n_steps + k]) - m);
            t += w[s];
        }
        for (int s = 0; s < n_sec; ++s) w[s] /= t;
        return m + std::log(t);
    };
    double m0 = -INFINITY, t0 = 0;
    for (int s = 0; s < n_sec; ++s) m0 = std::max(m0, 2.0 * lognorm0[s]);
    for (int s = 0; s < n_sec; ++s) t0 += std::exp(2.0 * lognorm0[s] - m0);
    const double l0 = m0 + std::log(t0);
    std::vector<double> w;
    for (int k = 0; k < n_steps; ++k) {
        const double lk = lse2(k, w);
        logQ_out[k] = 0.5 * (lk - l0);
        double uu = 0;
        for (int s = 0; s < n_sec; ++s) uu += w[s] * u[(size_t)s * n_steps + k];
        u_out[k] = uu;
    }
    for (int sh = 0; sh < n_shell; ++sh) {
        const int k = shell_steps[sh];
        if (k < 0 || k >= n_steps) {
            set_thread_error("ftk_sector_combine: shell step out of range");
            return FTK_EINVAL;
        }
        lse2(k, w);
        for (int o = 0; o < 2 * n_omega; ++o) {
            double acc = 0;
            for (int s = 0; s < n_sec; ++s) acc += w[s] * G[((size_t)s * n_shell + sh) * 2 * n_omega + o];
            G_out[(size_t)sh * 2 * n_omega + o] = acc;
        }
    }
    return FTK_OK;
}

}  // extern "C"
