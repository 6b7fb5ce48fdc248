// Device helpers shared by the FTKomega kernels: complex element types,
// per-thread dot accumulators and deterministic block / last-block
// reductions (fixed summation order, no floating-point atomics).
#pragma once
#include "ftk_common.cuh"

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
// The error-free steps are written with the rounded intrinsics (__fadd_rn,
// __fmul_rn, which the compiler never contracts into an FMA): a contracted
// t = s + a b would no longer be the rounded sum the two-sum corrects.
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
template <> struct Acc<float> {
    float s, c;
    __device__ Acc() : s(0.f), c(0.f) {}
    __device__ __forceinline__ void add(float v) {
        const float t = fadd(s, v);
        const float bp = fsub(t, s);
        const float err = fadd(fsub(s, fsub(t, bp)), fsub(v, bp));
        s = t;
        c = fadd(c, err);
    }
    __device__ __forceinline__ void fma2(float a, float b) {
        const float p = fmul(a, b);
        const float e = fmaf(a, b, -p);
        add(p);
        c = fadd(c, e);
    }
    // adds (ah + al)(bh + bl): the hi x hi product exactly (FMA two-product),
    // the cross terms in float (their lo x lo term is below the pair precision)
    __device__ __forceinline__ void fma_pair(float ah, float al, float bh, float bl) {
        const float p = fmul(ah, bh);
        float e = fmaf(ah, bh, -p);
        e = fmaf(ah, bl, e);
        e = fmaf(al, bh, e);
        add(p);
        c = fadd(c, e);
    }
    // adds (ah + al) b
    __device__ __forceinline__ void fma_hl(float ah, float al, float b) {
        const float p = fmul(ah, b);
        float e = fmaf(ah, b, -p);
        e = fmaf(al, b, e);
        add(p);
        c = fadd(c, e);
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

}  // namespace ftk

// ------------------------------------------------------------ double-float
// Unevaluated sums hi + lo of two floats (Dekker 1971; Knuth's two-sum, the
// FMA two-product): about 48 significant bits on the FP32 pipe, which on
// GB300 issues 64x the FP64 rate. The mixed mode stores its Krylov residuals
// as such pairs and updates them in this arithmetic.
namespace ftk {

struct dfl { float hi, lo; };

// Device only, with the rounded intrinsics of Acc<float> (no contraction).
__device__ __forceinline__ dfl dfl_two_sum(float a, float b) {
    const float s = fadd(a, b);
    const float bb = fsub(s, a);
    return {s, fadd(fsub(a, fsub(s, bb)), fsub(b, bb))};
}
__device__ __forceinline__ dfl dfl_fast(float a, float b) {   // |a| >= |b| or a == 0
    const float s = fadd(a, b);
    return {s, fsub(b, fsub(s, a))};
}
__device__ __forceinline__ dfl dfl_add(dfl a, dfl b) {
    const dfl s = dfl_two_sum(a.hi, b.hi);
    return dfl_fast(s.hi, fadd(s.lo, fadd(a.lo, b.lo)));
}
__device__ __forceinline__ dfl dfl_neg(dfl a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dfl dfl_sub(dfl a, dfl b) { return dfl_add(a, dfl_neg(b)); }
__device__ __forceinline__ dfl dfl_mul(dfl a, dfl b) {
    const float p = fmul(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return dfl_fast(p, e);
}
__device__ __forceinline__ dfl dfl_from(double d) {
    const float h = (float)d;
    return {h, (float)(d - (double)h)};
}

struct dcl { dfl re, im; };
__device__ __forceinline__ dcl dcl_add(dcl a, dcl b) { return {dfl_add(a.re, b.re), dfl_add(a.im, b.im)}; }
__device__ __forceinline__ dcl dcl_sub(dcl a, dcl b) { return {dfl_sub(a.re, b.re), dfl_sub(a.im, b.im)}; }
__device__ __forceinline__ dcl dcl_mul(dcl a, dcl b) {
    return {dfl_sub(dfl_mul(a.re, b.re), dfl_mul(a.im, b.im)), dfl_add(dfl_mul(a.re, b.im), dfl_mul(a.im, b.re))};
}

// ------------------------------------------------ COCG residual, split form
// The scalars of one COCG step for one right-hand side as double-float
// pairs: a1 = 1 + c_k - alpha_k z_s (formed in FP64 by the seed kernel),
// alpha_k, c_k, and the range-guard factor f (a power of two, 1 when unused).
struct DfStep {
    dcl a1, al, cc;
    float f;
};
__device__ __forceinline__ DfStep df_step(const CocgSeed &s) {
    return {{dfl_from(s.a1_re), dfl_from(s.a1_im)}, {dfl_from(s.alpha_re), dfl_from(s.alpha_im)},
            {dfl_from(s.c_re), dfl_from(s.c_im)}, (float)s.rescale};
}
// acc += a b in double-float: the hi x hi product exactly (FMA two-product)
// plus the cross terms, added by a two-sum whose error goes to acc.lo (the
// lo x lo term is below the pair precision). 12 FP32 operations.
__device__ __forceinline__ void dfl_mac(dfl &acc, dfl a, dfl b) {
    const float p = fmul(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float t = fadd(acc.hi, p);
    const float bb = fsub(t, acc.hi);
    acc.lo = fadd(acc.lo, fadd(fadd(fsub(acc.hi, fsub(t, bb)), fsub(p, bb)), e));
    acc.hi = t;
}
// Renormalised pair of an accumulator (two-sum: no ordering assumption).
__device__ __forceinline__ dfl dfl_renorm(dfl a) { return dfl_two_sum(a.hi, a.lo); }

// Three-term COCG residual (Sec. IV): with w_k = H r_k,
// r_{k+1} = r_k + c_k (r_k - r_{k-1}) - alpha_k (z_s r_k - w_k)
//         = a1 r_k - c_k r_{k-1} + alpha_k w_k,   a1 = 1 + c_k - alpha_k z_s,
// scaled by f. Each real component is the double-float sum of six products
// (the first one exact, then multiply-accumulates), renormalised once; its
// rounding error is bounded by 2^-48 (|a1| |r_k| + |c_k| |r_{k-1}| +
// |alpha_k| |w_k|), no more than that of forming z_s r_k - w_k and
// r_k - r_{k-1} first.
__device__ __forceinline__ dcl df_next_residual(const dcl &rc, const dcl &rp, const dcl &w, const DfStep &q) {
    dfl nr = dfl_mul(q.a1.re, rc.re);
    dfl_mac(nr, dfl_neg(q.a1.im), rc.im);
    dfl_mac(nr, dfl_neg(q.cc.re), rp.re);
    dfl_mac(nr, q.cc.im, rp.im);
    dfl_mac(nr, q.al.re, w.re);
    dfl_mac(nr, dfl_neg(q.al.im), w.im);
    dfl ni = dfl_mul(q.a1.re, rc.im);
    dfl_mac(ni, q.a1.im, rc.re);
    dfl_mac(ni, dfl_neg(q.cc.re), rp.im);
    dfl_mac(ni, dfl_neg(q.cc.im), rp.re);
    dfl_mac(ni, q.al.re, w.im);
    dfl_mac(ni, q.al.im, w.re);
    nr = dfl_renorm(nr);
    ni = dfl_renorm(ni);
    if (q.f != 1.f) { nr = {fmul(nr.hi, q.f), fmul(nr.lo, q.f)}; ni = {fmul(ni.hi, q.f), fmul(ni.lo, q.f)}; }
    return {nr, ni};
}
// Per-thread sums of rho = r^T r, g = lambda^dag r (double-float: exact
// two-products of the hi parts plus cross terms, two-sums) and |r|^2 (float
// of the hi parts: only the convergence test and the range guard read it).
// l4 = (lambda hi.re, hi.im, lo.re, lo.im).
struct DfUpdDots {
    Acc<float> rr, ri, gr, gi;
    float n = 0.f;
    __device__ __forceinline__ void add(const dcl &r, const float4 &l4) {
        rr.fma_pair(r.re.hi, r.re.lo, r.re.hi, r.re.lo);
        rr.fma_pair(-r.im.hi, -r.im.lo, r.im.hi, r.im.lo);
        ri.fma_pair(2.f * r.re.hi, 2.f * r.re.lo, r.im.hi, r.im.lo);
        gr.fma_pair(l4.x, l4.z, r.re.hi, r.re.lo);
        gr.fma_pair(l4.y, l4.w, r.im.hi, r.im.lo);
        gi.fma_pair(l4.x, l4.z, r.im.hi, r.im.lo);
        gi.fma_pair(-l4.y, -l4.w, r.re.hi, r.re.lo);
        n = fmaf(r.re.hi, r.re.hi, fmaf(r.im.hi, r.im.hi, n));
    }
    __device__ __forceinline__ void get(double (&v)[5]) const {
        v[0] = rr.get(); v[1] = ri.get(); v[2] = gr.get(); v[3] = gi.get(); v[4] = n;
    }
};

}  // namespace ftk
