// Host runtime and C-ABI of the FTKomega hot path: context, H.v pass planner,
// workspace carving, CUDA-graph captured Krylov chunks, autotuned tiles.
#include "../../include/ftk.h"
#include "ftk_common.cuh"
#include "ftk_kernels.h"
#include "ftk_plan.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

using namespace ftk;

namespace {

const size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Bond { int i, j, g; };

// Workspace regions (bytes from the workspace base).
struct Layout {
    size_t psi[2], shells, probes, kry[3], lam_split, partials, shift, omega, gbuf, tbuf, total;
    size_t vec_bytes;
};

const size_t kPartialsBytes = size_t(4) << 20;
const int kShiftArrays = 5;

Layout make_layout(int n, int n_saved, int max_rhs, int prec) {
    Layout L{};
    const size_t es = prec == FTK_FP32 ? 8 : 16;   // FTK_MIXED stores FP64 vectors
    const size_t vb = (size_t(1) << n) * es;
    size_t off = 0;
    L.vec_bytes = vb;
    // the mTPQ state is always FP64 (16 B / amplitude); shells, probes and
    // Krylov vectors use the context's vector precision
    const size_t vb64 = (size_t(1) << n) * 16;
    for (int i = 0; i < 2; ++i) { L.psi[i] = off; off = align_up(off + vb64); }
    L.shells = off; off = align_up(off + vb * n_saved);
    L.probes = off; off = align_up(off + vb * max_rhs);
    for (int i = 0; i < 3; ++i) { L.kry[i] = off; off = align_up(off + vb * max_rhs); }
    // mixed and double-float modes: the probe vectors split into float hi + lo
    L.lam_split = off;
    if (prec == FTK_MIXED || prec == FTK_DF) off = align_up(off + (size_t(1) << n) * 16 * max_rhs);
    L.partials = off; off = align_up(off + kPartialsBytes);
    L.shift = off; off = align_up(off + size_t(kShiftArrays) * max_rhs * FTK_MAX_OMEGA * 16);
    L.omega = off; off = align_up(off + FTK_MAX_OMEGA * 16);   // complex shift offsets
    L.gbuf = off; off = align_up(off + size_t(1024) * FTK_MAX_OMEGA * 16);   // spectrum input G
    L.tbuf = off; off = align_up(off + 3 * 1024 * 8);          // T; shell energies and norms
    L.total = off;
    return L;
}

// Small device buffers owned by the context.
struct Small {
    TpqState tpq;
    unsigned int counters[8];
    double hv_dots[FTK_MAX_RHS * FTK_HV_DOTS];
    double upd_dots[FTK_MAX_RHS * FTK_UPD_DOTS];
    double op_dots[4];
    double inv_pi_max[2 * FTK_MAX_RHS];
    int all_done;
    int lowp;                        // relaxed solve: FP32 products from here on
    CocgSeed seed[FTK_MAX_RHS];
};

struct Plan {
    int tile_bits = 0, chunk_bits = 0, threads = 512, grid = 0;
    size_t smem = 0;
    std::vector<PassDesc> passes;
};

}  // namespace

namespace ftk {
void set_thread_error(const char *msg);
}

struct ftk_ctx {
    int n = 0, nb = 0, prec = 0, max_rhs = 1, n_saved_cap = 1, tile_bits_req = 0;
    int vprec = 0, mprec = 0;   // vector storage / H.v arithmetic: 0 FP64, 1 FP32
    double relax = 0.0;         // relaxed double-float solve: theta (0: off)
    uint64_t dim = 0;
    double K = 0, J = 0, ell_min = 0;
    std::vector<Bond> bonds;
    std::vector<double> pos;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int n_sm = 0, device = 0;
    Small *dsmall = nullptr;         // device
    double *stats = nullptr;         // device [3][cap]: u, logq, h2
    int stats_cap = 0;
    double *shell_scale = nullptr;   // device [n_saved_cap]
    double *slot_energy = nullptr;   // device [max_rhs]
    double *slot_norm2 = nullptr;    // device [max_rhs]
    char *ws = nullptr;
    size_t ws_bytes = 0;
    Layout L{};
    // host mirrors
    int k = 0, n_saved = 0, save_every = 1, have_state = 0;
    double ell = 0.5;
    std::vector<int> shell_step;
    // shift origin of shells not produced by the mTPQ iteration (cTPQ and
    // filtered shells); NaN: an mTPQ shell, origin N u_k from the statistics
    std::vector<double> shell_origin;
    cudaGraphExec_t cocg_exec = nullptr;   // instantiated COCG graph of the last solve
    std::vector<int> slot_valid;
    std::map<int, Plan> plans;       // by (precision, block width B): key prec * 64 + B
    int64_t launches = 0;
    std::string err;
};

namespace {

thread_local std::string g_create_err;   // last context-free failure on this thread

ftk_status fail(ftk_ctx *c, ftk_status s, const std::string &m) {
    if (c) c->err = m;
    else g_create_err = m;
    return s;
}

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(ctx, FTK_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define LAUNCH(call)        \
    do {                    \
        CK(call);           \
        ++ctx->launches;    \
    } while (0)

int elem_bytes(int prec) { return prec == 1 ? 8 : 16; }   // H.v arithmetic: 0 FP64, 1 FP32, 2 double-float

}  // namespace

void ftk::set_thread_error(const char *msg) { g_create_err = msg; }

namespace {

// Plan the passes of H.V for column chunks of bc right-hand sides: the
// planner with its local search first; if that plan cannot be laid out for
// the kernel (or needs too much shared memory), the greedy plan alone.
bool plan_passes_with(ftk_ctx *ctx, int prec, int bc, int tile_bits, long local_steps, Plan &pl) {
    PlanBond pb[2 * FTK_MAX_PASS_BONDS];
    for (int q = 0; q < ctx->nb; ++q) pb[q] = {ctx->bonds[q].i, ctx->bonds[q].j, ctx->bonds[q].g};
    PassDesc pd[FTK_MAX_PASSES];
    const int np = plan_hv_passes(ctx->n, pb, ctx->nb, ctx->K, ctx->J, elem_bytes(prec), bc, tile_bits, pd,
                                  FTK_MAX_PASSES, &pl.tile_bits, &pl.chunk_bits, 32, local_steps);
    if (np == 0) return false;
    for (int p = 0; p < np; ++p)
        if (!hv_layout_pass(pd[p], prec, bc)) return false;
    pl.passes.assign(pd, pd + np);
    pl.threads = hv_threads(pl.passes[0]);
    pl.smem = hv_smem_bytes(prec, bc, pl.passes[0]);
    pl.grid = 8 * ctx->n_sm;   // cap of the persistent grid (4 MB of reduction partials)
    return pl.smem <= (size_t(227) << 10);
}

bool plan_passes(ftk_ctx *ctx, int prec, int bc, int tile_bits, Plan &pl) {
    if (plan_passes_with(ctx, prec, bc, tile_bits, kPlanLocalSteps, pl)) return true;
    pl = Plan{};
    return plan_passes_with(ctx, prec, bc, tile_bits, 0, pl);
}

ftk_status get_plan(ftk_ctx *ctx, int prec, int B, Plan **out) {
    auto it = ctx->plans.find(prec * 64 + B);
    if (it != ctx->plans.end()) { *out = &it->second; return FTK_OK; }
    // default: all columns in one launch (at most hv_max_b), the largest tile;
    // the FP32 products of a relaxed double-float solve: one column per
    // launch (the largest tile, fewest passes)
    const int bc = (prec == FTK_FP32 && ctx->prec == FTK_DF) ? 1 : std::min(B, hv_max_b(prec));
    const int tb_max = hv_max_tile_bits(prec, bc);
    int tb = ctx->tile_bits_req > 0 ? std::min(ctx->tile_bits_req, tb_max) : tb_max;
    tb = std::max(2, std::min(tb, ctx->n));
    Plan pl;
    if (!plan_passes(ctx, prec, bc, tb, pl))
        return fail(ctx, FTK_EINVAL, "H.v pass planning failed (tile too small for the bond list)");
    auto res = ctx->plans.emplace(prec * 64 + B, pl);
    *out = &res.first->second;
    return FTK_OK;
}

char *wsp(ftk_ctx *ctx, size_t off) { return ctx->ws + off; }

int vec_grid(ftk_ctx *ctx, uint64_t n_items) {
    const uint64_t want = (n_items + 255) / 256;
    const uint64_t cap = uint64_t(4) * ctx->n_sm;
    return (int)std::max<uint64_t>(1, std::min(want, cap));
}

// H.V over all passes. The last pass uses epilogue epi, earlier ones write
// or accumulate the partial product into out.
ftk_status run_hv(ftk_ctx *ctx, int prec, int B, int epi, const void *in, void *out, EpiArgs ea) {
    Plan *pl = nullptr;
    ftk_status s = get_plan(ctx, prec, B, &pl);
    if (s != FTK_OK) return s;
    const int np = (int)pl->passes.size();
    for (int p = 0; p < np; ++p) {
        const int e = (p == np - 1) ? epi : EPI_PLAIN;
        LAUNCH(launch_hv_pass(prec, B, e, in, out, pl->passes[p], ea, pl->grid, ctx->stream));
    }
    return FTK_OK;
}

// One process-wide lock for the device calls that synchronise the whole
// device (cudaMalloc / cudaFree of the context buffers) and for the capture
// window of the COCG graph: contexts of different host threads (the server
// runs one per job) must not free or allocate while another thread's stream
// is being captured.
std::mutex &device_mu() {
    static std::mutex m;
    return m;
}

ftk_status ensure_stats(ftk_ctx *ctx, int need) {
    if (need <= ctx->stats_cap) return FTK_OK;
    std::lock_guard<std::mutex> lk(device_mu());
    int cap = std::max(need, std::max(1024, ctx->stats_cap * 2));
    double *nb = nullptr;
    CK(cudaMalloc(&nb, size_t(3) * cap * sizeof(double)));
    CK(cudaMemsetAsync(nb, 0, size_t(3) * cap * sizeof(double), ctx->stream));
    if (ctx->stats) {
        for (int a = 0; a < 3; ++a)
            CK(cudaMemcpyAsync(nb + size_t(a) * cap, ctx->stats + size_t(a) * ctx->stats_cap,
                               ctx->stats_cap * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        cudaFree(ctx->stats);
    }
    ctx->stats = nb;
    ctx->stats_cap = cap;
    return FTK_OK;
}

double *stat_u(ftk_ctx *c) { return c->stats; }
double *stat_lq(ftk_ctx *c) { return c->stats + c->stats_cap; }
double *stat_h2(ftk_ctx *c) { return c->stats + 2 * size_t(c->stats_cap); }

ftk_status check_ready(ftk_ctx *ctx) {
    if (!ctx) return FTK_EINVAL;
    if (!ctx->ws) return fail(ctx, FTK_ENOMEM, "no workspace bound");
    return FTK_OK;
}

// A shell slot below n_saved that holds a state: an mTPQ shell (step >= 0)
// or a cTPQ / filtered shell (its origin set). Slots skipped by a
// first_shell > n_saved are not written.
bool shell_written(const ftk_ctx *ctx, int s) {
    return s >= 0 && s < ctx->n_saved && (ctx->shell_step[s] >= 0 || !std::isnan(ctx->shell_origin[s]));
}

ftk_status check_ell(ftk_ctx *ctx, double ell) {
    if (!(ell >= ctx->ell_min - 1e-12))
        return fail(ctx, FTK_EINVAL, "ell below l_min = (1/N) sum_b lambda_max(h_b) = " +
                                         std::to_string(ctx->ell_min));
    return FTK_OK;
}

}  // namespace

// Hamiltonian and stream of a context for the momentum-sector code.
bool ftk::ctx_hamiltonian(ftk_ctx *c, CtxHam *h) {
    if (!c) return false;
    h->n = c->n;
    h->nb = c->nb;
    h->bonds = reinterpret_cast<const int *>(c->bonds.data());
    h->K = c->K;
    h->J = c->J;
    h->ell_min = c->ell_min;
    h->pos = c->pos.data();
    h->stream = c->stream;
    h->n_sm = c->n_sm;
    h->launches = &c->launches;
    h->err = &c->err;
    return true;
}

extern "C" {

size_t ftk_footprint(int32_t n_sites, int32_t n_saved, int32_t max_rhs, int32_t precision) {
    if (n_sites < 2 || n_sites > FTK_MAX_SITES || n_saved < 1 || max_rhs < 1 ||
        max_rhs > FTK_MAX_RHS || precision < FTK_FP64 || precision > FTK_DF)
        return 0;
    return make_layout(n_sites, n_saved, max_rhs, precision).total;
}

ftk_status ftk_create(const ftk_lattice *lat, const ftk_bond *bonds, int32_t n_bonds, double K,
                      double J, const ftk_opts *opts, ftk_ctx **out) {
    if (!out) return fail(nullptr, FTK_EINVAL, "null output handle");
    *out = nullptr;
    if (!lat || !bonds || !opts || !lat->pos) return fail(nullptr, FTK_EINVAL, "null argument");
    const int n = lat->n_sites;
    if (n < 2 || n > FTK_MAX_SITES) return fail(nullptr, FTK_EINVAL, "n_sites must be in [2, 30]");
    if (n_bonds < 1 || n_bonds > 2 * FTK_MAX_PASS_BONDS) return fail(nullptr, FTK_EINVAL, "bad n_bonds");
    if (opts->precision < FTK_FP64 || opts->precision > FTK_DF)
        return fail(nullptr, FTK_EINVAL, "precision must be FTK_FP64, FTK_FP32, FTK_MIXED or FTK_DF");
    if (opts->max_rhs < 1 || opts->max_rhs > FTK_MAX_RHS || opts->n_saved < 1)
        return fail(nullptr, FTK_EINVAL, "max_rhs must be in [1, 32] and n_saved >= 1");
    if (!std::isfinite(K) || !std::isfinite(J)) return fail(nullptr, FTK_EINVAL, "K, J must be finite");
    for (int q = 0; q < n_bonds; ++q) {
        const ftk_bond &b = bonds[q];
        if (b.i < 0 || b.j < 0 || b.i >= n || b.j >= n || b.i == b.j || b.gamma < 0 || b.gamma > 2)
            return fail(nullptr, FTK_EINVAL, "bond " + std::to_string(q) + " out of range");
    }
    ftk_ctx *ctx = new (std::nothrow) ftk_ctx();
    if (!ctx) return FTK_ENOMEM;
    ctx->n = n;
    ctx->nb = n_bonds;
    ctx->dim = uint64_t(1) << n;
    ctx->K = K;
    ctx->J = J;
    ctx->prec = opts->precision;
    ctx->vprec = ctx->prec == FTK_FP32 ? 1 : 0;
    ctx->mprec = ctx->prec == FTK_FP64 ? 0 : ctx->prec == FTK_DF ? 2 : 1;
    ctx->max_rhs = opts->max_rhs;
    ctx->n_saved_cap = opts->n_saved;
    ctx->tile_bits_req = opts->tile_bits;
    ctx->pos.assign(lat->pos, lat->pos + 2 * n);
    for (int q = 0; q < n_bonds; ++q) ctx->bonds.push_back({bonds[q].i, bonds[q].j, bonds[q].gamma});
    // l_min: the bond block has eigenvalues (J+K)/4 (x2), (J-K)/4, -(3J+K)/4
    const double lmax = std::max({(J + K) / 4, (J - K) / 4, -(3 * J + K) / 4});
    ctx->ell_min = n_bonds * lmax / n;
    ctx->slot_valid.assign(ctx->max_rhs, 0);
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e != cudaSuccess) { delete ctx; return fail(nullptr, FTK_ECUDA, cudaGetErrorString(e)); }
    if (opts->cuda_stream) {
        ctx->stream = (cudaStream_t)opts->cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete ctx; return fail(nullptr, FTK_ECUDA, cudaGetErrorString(e)); }
        ctx->own_stream = true;
    }
    std::unique_lock<std::mutex> lk(device_mu());
    e = cudaMalloc(&ctx->dsmall, sizeof(Small));
    if (e == cudaSuccess) e = cudaMemset(ctx->dsmall, 0, sizeof(Small));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->shell_scale, sizeof(double) * ctx->n_saved_cap);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->slot_energy, sizeof(double) * ctx->max_rhs);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->slot_norm2, sizeof(double) * ctx->max_rhs);
    const cudaError_t ka = e == cudaSuccess ? init_kernel_attributes() : cudaSuccess;
    lk.unlock();   // ftk_destroy takes the lock itself
    if (e != cudaSuccess) { ftk_destroy(ctx); return fail(nullptr, FTK_ECUDA, cudaGetErrorString(e)); }
    if (ka != cudaSuccess) {
        ftk_destroy(ctx);
        return fail(nullptr, FTK_ECUDA, std::string("kernel attributes: ") + cudaGetErrorString(ka));
    }
    Plan *pl = nullptr;
    if (get_plan(ctx, ctx->mprec, 1, &pl) != FTK_OK) {
        std::string m = ctx->err;
        ftk_destroy(ctx);
        return fail(nullptr, FTK_EINVAL, m);
    }
    *out = ctx;
    return FTK_OK;
}

ftk_status ftk_bind_workspace(ftk_ctx *ctx, void *dev_ptr, size_t bytes) {
    if (!ctx) return FTK_EINVAL;
    if (!dev_ptr || (reinterpret_cast<uintptr_t>(dev_ptr) % kAlign) != 0)
        return fail(ctx, FTK_EINVAL, "workspace must be non-null and 256-byte aligned");
    Layout L = make_layout(ctx->n, ctx->n_saved_cap, ctx->max_rhs, ctx->prec);
    if (bytes < L.total)
        return fail(ctx, FTK_ENOMEM, "workspace too small: need " + std::to_string(L.total));
    ctx->ws = (char *)dev_ptr;
    ctx->ws_bytes = bytes;
    ctx->L = L;
    ctx->have_state = 0;
    ctx->n_saved = 0;
    ctx->k = 0;
    ctx->slot_valid.assign(ctx->max_rhs, 0);
    CK(cudaMemsetAsync(ctx->dsmall, 0, sizeof(Small), ctx->stream));
    return FTK_OK;
}

ftk_status ftk_tpq_init(ftk_ctx *ctx, uint64_t seed, uint32_t sample, double ell) {
    ftk_status s = check_ready(ctx);
    if (s) return s;
    if ((s = check_ell(ctx, ell))) return s;
    ctx->ell = ell;
    InitArgs ia{};
    ia.dim = ctx->dim;
    ia.seed = seed;
    ia.sample = sample;
    ia.partials = (double *)wsp(ctx, ctx->L.partials);
    ia.counter = &ctx->dsmall->counters[0];
    ia.result = ctx->dsmall->op_dots;
    ia.tpq = &ctx->dsmall->tpq;
    TpqState h{};
    h.ell = ell;
    h.n_sites = ctx->n;
    CK(cudaMemcpyAsync(&ctx->dsmall->tpq, &h, sizeof h, cudaMemcpyHostToDevice, ctx->stream));
    LAUNCH(launch_init_state(FTK_FP64, wsp(ctx, ctx->L.psi[0]), ia, vec_grid(ctx, ctx->dim), ctx->stream));
    ctx->k = 0;
    ctx->n_saved = 0;
    ctx->have_state = 1;
    return FTK_OK;
}

static ftk_status load_vector(ftk_ctx *ctx, const double *v, int is_device, void *dst, int prec) {
    // stage as double2 in the Krylov region (3 * max_rhs vectors >= 16 B / amplitude)
    void *stage = wsp(ctx, ctx->L.kry[0]);
    const size_t bytes = ctx->dim * 16;
    if (prec == FTK_FP64) {
        CK(cudaMemcpyAsync(dst, v, bytes, is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           ctx->stream));
        return FTK_OK;
    }
    CK(cudaMemcpyAsync(stage, v, bytes, is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       ctx->stream));
    LAUNCH(launch_convert_in(prec, stage, dst, ctx->dim, vec_grid(ctx, ctx->dim), ctx->stream));
    return FTK_OK;
}

ftk_status ftk_set_state(ftk_ctx *ctx, const double *v, int32_t is_device, double ell) {
    ftk_status s = check_ready(ctx);
    if (s) return s;
    if (!v) return fail(ctx, FTK_EINVAL, "null vector");
    if ((s = check_ell(ctx, ell))) return s;
    ctx->ell = ell;
    TpqState h{};
    h.ell = ell;
    h.n_sites = ctx->n;
    CK(cudaMemcpyAsync(&ctx->dsmall->tpq, &h, sizeof h, cudaMemcpyHostToDevice, ctx->stream));
    if ((s = load_vector(ctx, v, is_device, wsp(ctx, ctx->L.psi[0]), FTK_FP64))) return s;
    InitArgs ia{};
    ia.dim = ctx->dim;
    ia.partials = (double *)wsp(ctx, ctx->L.partials);
    ia.counter = &ctx->dsmall->counters[0];
    ia.result = ctx->dsmall->op_dots;
    ia.tpq = &ctx->dsmall->tpq;
    LAUNCH(launch_norm(FTK_FP64, wsp(ctx, ctx->L.psi[0]), ia, vec_grid(ctx, ctx->dim), ctx->stream));
    ctx->k = 0;
    ctx->n_saved = 0;
    ctx->have_state = 1;
    if (!is_device) CK(cudaStreamSynchronize(ctx->stream));
    return FTK_OK;
}

ftk_status ftk_tpq_step(ftk_ctx *ctx, int32_t n_steps, int32_t save_every, double *u_out,
                        double *logQ_out, double *h2_out) {
    ftk_status s = check_ready(ctx);
    if (s) return s;
    if (!ctx->have_state) return fail(ctx, FTK_EBUSY, "no TPQ state: call ftk_tpq_init first");
    Plan *pl64 = nullptr;
    if ((s = get_plan(ctx, FTK_FP64, 1, &pl64))) return s;
    if (n_steps < 0 || save_every < 1) return fail(ctx, FTK_EINVAL, "bad n_steps / save_every");
    if (ctx->n_saved > 0 && save_every != ctx->save_every)
        return fail(ctx, FTK_EINVAL, "save_every must not change between calls");
    ctx->save_every = save_every;
    const int k0 = ctx->k;
    int need_saved = ctx->n_saved;
    for (int k = k0; k < k0 + n_steps; ++k) need_saved += (k % save_every == 0);
    if (need_saved > ctx->n_saved_cap)
        return fail(ctx, FTK_ENOMEM, "more shells than n_saved (" + std::to_string(ctx->n_saved_cap) + ")");
    if ((s = ensure_stats(ctx, k0 + n_steps))) return s;
    EpiArgs ea{};
    ea.scale = &ctx->dsmall->tpq.scale;
    ea.ell = ctx->ell;
    ea.inv_n = 1.0 / ctx->n;
    ea.partials = (double *)wsp(ctx, ctx->L.partials);
    ea.counter = &ctx->dsmall->counters[1];
    ea.result = ctx->dsmall->op_dots;
    ea.tpq = &ctx->dsmall->tpq;
    ea.stat_u = stat_u(ctx);
    ea.stat_logq = stat_lq(ctx);
    ea.stat_h2 = stat_h2(ctx);
    for (int k = k0; k < k0 + n_steps; ++k) {
        void *cur = wsp(ctx, ctx->L.psi[k & 1]);
        void *nxt = wsp(ctx, ctx->L.psi[(k + 1) & 1]);
        if (k % save_every == 0) {
            const int sidx = ctx->n_saved;
            void *dst = wsp(ctx, ctx->L.shells + ctx->L.vec_bytes * sidx);
            if (ctx->vprec == 0)
                CK(cudaMemcpyAsync(dst, cur, ctx->L.vec_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
            else
                LAUNCH(launch_convert_in(ctx->vprec, cur, dst, ctx->dim, vec_grid(ctx, ctx->dim), ctx->stream));
            CK(cudaMemcpyAsync(ctx->shell_scale + sidx, &ctx->dsmall->tpq.scale, sizeof(double),
                               cudaMemcpyDeviceToDevice, ctx->stream));
            ctx->shell_step.resize(sidx + 1);
            ctx->shell_step[sidx] = k;
            ctx->shell_origin.resize(sidx + 1);
            ctx->shell_origin[sidx] = NAN;
            ctx->n_saved = sidx + 1;
        }
        if ((s = run_hv(ctx, FTK_FP64, 1, EPI_TPQ, cur, nxt, ea))) return s;
        ctx->k = k + 1;
    }
    CK(cudaStreamSynchronize(ctx->stream));
    if (n_steps > 0) {
        if (u_out) CK(cudaMemcpyAsync(u_out, stat_u(ctx) + k0, n_steps * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        if (logQ_out)
            CK(cudaMemcpyAsync(logQ_out, stat_lq(ctx) + k0, n_steps * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        if (h2_out) CK(cudaMemcpyAsync(h2_out, stat_h2(ctx) + k0, n_steps * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return FTK_OK;
}

ftk_status ftk_shells(const ftk_ctx *cctx, int32_t *n_out, int32_t *step_out, double *energy_out) {
    ftk_ctx *ctx = const_cast<ftk_ctx *>(cctx);
    if (!ctx) return FTK_EINVAL;
    if (n_out) *n_out = ctx->n_saved;
    CK(cudaStreamSynchronize(ctx->stream));
    for (int s = 0; s < ctx->n_saved; ++s) {
        if (step_out) step_out[s] = ctx->shell_step[s];
        if (energy_out && !std::isnan(ctx->shell_origin[s])) {
            energy_out[s] = ctx->shell_origin[s];   // cTPQ or filtered shell: its origin
        } else if (energy_out && !shell_written(ctx, s)) {
            energy_out[s] = NAN;                    // slot not written
        } else if (energy_out) {
            double u = 0;
            CK(cudaMemcpyAsync(&u, stat_u(ctx) + ctx->shell_step[s], sizeof u, cudaMemcpyDeviceToHost, ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
            energy_out[s] = u * ctx->n;
        }
    }
    return FTK_OK;
}

ftk_status ftk_apply_op(ftk_ctx *ctx, int32_t shell, int32_t gamma, const double q[2], int32_t slot) {
    ftk_status s = check_ready(ctx);
    if (s) return s;
    if (!shell_written(ctx, shell)) return fail(ctx, FTK_EINVAL, "shell index out of range or not written");
    if (gamma < 0 || gamma > 2 || !q) return fail(ctx, FTK_EINVAL, "bad gamma or q");
    if (slot < 0 || slot >= ctx->max_rhs) return fail(ctx, FTK_EINVAL, "rhs slot out of range");
    const bool tpq_shell = std::isnan(ctx->shell_origin[shell]);
    if (tpq_shell && ctx->shell_step[shell] >= ctx->k)
        return fail(ctx, FTK_EBUSY, "shell statistics not computed yet (run one more TPQ step)");
    OpArgs oa{};
    oa.n_sites = ctx->n;
    oa.gamma = gamma;
    oa.dim = ctx->dim;
    const double nrm = 1.0 / std::sqrt((double)ctx->n);
    for (int l = 0; l < ctx->n; ++l) {
        const double ph = q[0] * ctx->pos[2 * l] + q[1] * ctx->pos[2 * l + 1];
        oa.f_re[l] = nrm * std::cos(ph);
        oa.f_im[l] = nrm * std::sin(ph);
    }
    oa.scale = ctx->shell_scale + shell;
    oa.partials = (double *)wsp(ctx, ctx->L.partials);
    oa.counter = &ctx->dsmall->counters[2];
    oa.result = ctx->dsmall->op_dots;
    oa.energy_src = tpq_shell ? stat_u(ctx) + ctx->shell_step[shell] : nullptr;
    oa.energy_val = tpq_shell ? 0.0 : ctx->shell_origin[shell];
    oa.n_sites_d = ctx->n;
    oa.slot_energy = ctx->slot_energy + slot;
    oa.slot_norm2 = ctx->slot_norm2 + slot;
    LAUNCH(launch_apply_op(ctx->vprec, wsp(ctx, ctx->L.shells + ctx->L.vec_bytes * shell),
                           wsp(ctx, ctx->L.probes + ctx->L.vec_bytes * slot), oa, vec_grid(ctx, ctx->dim),
                           ctx->stream));
    ctx->slot_valid[slot] = 1;
    return FTK_OK;
}

ftk_status ftk_set_probe(ftk_ctx *ctx, int32_t slot, const double *v, int32_t is_device, double energy) {
    ftk_status s = check_ready(ctx);
    if (s) return s;
    if (slot < 0 || slot >= ctx->max_rhs || !v) return fail(ctx, FTK_EINVAL, "bad slot or vector");
    if ((s = load_vector(ctx, v, is_device, wsp(ctx, ctx->L.probes + ctx->L.vec_bytes * slot), ctx->vprec))) return s;
    CK(cudaMemcpyAsync(ctx->slot_energy + slot, &energy, sizeof energy, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->slot_valid[slot] = 1;
    return FTK_OK;
}

// One blocked COCG iteration on the context stream (no host sync):
// H R_cur -> W (+mu), seed scalars, shift recurrences, R_prev <- update. In
// the double-float mode the order is shifted by one step: R_prev <- update
// of the previous step inside the first pass of H R_prev -> W (+mu), seed
// scalars, shift recurrences (step 0 runs before the captured loop).
// Kind of the update kernel: 0 FP64 vectors, 1 FP32 vectors, 2 mixed (split
// float hi + lo residuals; hi at the buffer start, lo ua.lo_stride float2
// elements later).
static int upd_kind(const ftk_ctx *ctx) { return ctx->prec >= FTK_MIXED ? 2 : ctx->vprec; }

// Extra launches of one COCG iteration beyond the standard ones: the seed
// switch kernel (after the seed kernel) and the second-pass filter
// accumulation (after the shift kernel, before the update).
struct IterExtras {
    const SwitchArgs *sw;        // NULL: no seed switching
    const FilterAccArgs *acc;    // NULL: no accumulation
};

static ftk_status cocg_iteration(ftk_ctx *ctx, int B, void *rcur, void *rprev, void *w,
                                 EpiArgs ea, const SeedArgs &sa, const ShiftArgs &sh,
                                 UpdArgs ua, const IterExtras &ex) {
    auto after_seed = [&](void *rc, void *rp) -> ftk_status {
        if (ex.sw) {
            SwitchArgs a = *ex.sw;
            a.rcur = rc;
            a.rprev = rp;
            a.w = w;
            LAUNCH(launch_cocg_switch(a, B, vec_grid(ctx, ctx->dim), ctx->stream));
        }
        return FTK_OK;
    };
    if (ctx->prec == FTK_DF) {
        // double-float: the update r_{k-1} <- r_{k+1} of the previous step runs
        // inside the first pass of H r_{k+1} (rcur = r_k, rprev = r_{k-1})
        if (ctx->relax > 0.0) {
            // relaxed phase (device flag lowp): the update alone, then the
            // FP32 H.V of the hi parts with mu from hi + lo; the
            // double-float launches below return at once, and these while
            // lowp is 0
            const int *lowp = &ctx->dsmall->lowp;
            UpdArgs u = ua;
            u.mode = 1;
            u.w_lo = 0;   // w of the switching step is read without its lo part
            u.lowp = lowp;
            u.lowp_run = 1;
            LAUNCH(launch_cocg_update(upd_kind(ctx), B, rcur, w, rprev, u, vec_grid(ctx, ctx->dim), ctx->stream));
            EpiArgs e1 = ea;
            e1.lo = static_cast<const char *>(rprev) + size_t(8) * ua.lo_stride;
            e1.lowp = lowp;
            e1.lowp_run = 1;
            ftk_status s1 = run_hv(ctx, FTK_FP32, B, EPI_COCG, rprev, w, e1);
            if (s1) return s1;
            ea.lowp = lowp;
            ea.lowp_run = 0;
        }
        ea.df_lo = ua.lo_stride;
        ea.fu_seed = ua.seed;
        ea.fu_rcur = static_cast<float2 *>(rcur);
        ea.fu_lam = ua.lam_split;
        ea.fu_result = ua.result;
        ftk_status s = run_hv(ctx, ctx->mprec, B, EPI_COCG, rprev, w, ea);
        if (s) return s;
        LAUNCH(launch_cocg_seed(sa, ctx->stream));
        // the new r_k is the buffer rprev (written by the fused update), r_{k-1} is rcur
        if ((s = after_seed(rprev, rcur))) return s;
        LAUNCH(launch_cocg_shift(sh, B, ctx->stream));
        return FTK_OK;
    }
    if (ctx->prec == FTK_MIXED) ea.lo = static_cast<const char *>(rcur) + size_t(8) * ua.lo_stride;
    ftk_status s = run_hv(ctx, ctx->mprec, B, EPI_COCG, rcur, w, ea);
    if (s) return s;
    LAUNCH(launch_cocg_seed(sa, ctx->stream));
    if ((s = after_seed(rcur, rprev))) return s;
    LAUNCH(launch_cocg_shift(sh, B, ctx->stream));
    if (ex.acc) {
        FilterAccArgs a = *ex.acc;
        a.r = static_cast<const double2 *>(rcur);
        LAUNCH(launch_filter_acc(a, vec_grid(ctx, ctx->dim), ctx->stream));
    }
    ua.mode = 1;
    LAUNCH(launch_cocg_update(upd_kind(ctx), B, rcur, w, rprev, ua, vec_grid(ctx, ctx->dim), ctx->stream));
    return FTK_OK;
}

// One shifted-COCG solve of a block (the core of ftk_shifted_cocg,
// ftk_shifted_cocg_ex and the contour filter).
struct CocgReq {
    const int32_t *slots = nullptr;     // probe slots of the right-hand sides
    const int32_t *proj = nullptr;      // probe slots of the projection vectors (NULL: the rhs)
    int n_rhs = 0;
    const double *shift = nullptr;      // host [n_shift][2]: z_js - E_j
    int n_shift = 0;
    int seed_index = -1;                // -1: n_shift / 2
    int seed_switch = 0;
    double tol = 0;
    int max_iter = 0;
    dcx *hist = nullptr;                // device history (rhs 0), or NULL
    int hist_cap = 0;
    const FilterAccArgs *acc = nullptr; // second filter pass, or NULL
};

// Instantiated graph of the last solve; a later solve updates it in place
// (cudaGraphExecUpdate) when the captured launch sequence has the same shape,
// so repeated solves do not pay for a new instantiation.
static ftk_status instantiate_cached(ftk_ctx *ctx, cudaGraph_t graph, cudaGraphExec_t *out) {
    if (ctx->cocg_exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(ctx->cocg_exec, graph, &info) == cudaSuccess) {
            *out = ctx->cocg_exec;
            return FTK_OK;
        }
        (void)cudaGetLastError();   // a failed update leaves no sticky error
        cudaGraphExecDestroy(ctx->cocg_exec);
        ctx->cocg_exec = nullptr;
    }
    CK(cudaGraphInstantiate(&ctx->cocg_exec, graph, 0));
    *out = ctx->cocg_exec;
    return FTK_OK;
}

static ftk_status cocg_core(ftk_ctx *ctx, const CocgReq &rq, double *G_out, int32_t *iters_out,
                            int32_t *switches_out) {
    const int n_rhs = rq.n_rhs, n_omega = rq.n_shift;
    int B = 1;
    while (B < n_rhs) B <<= 1;
    if (B > ctx->max_rhs) {
        // block wider than the Krylov region: split into two halves
        if (rq.hist || rq.acc) return fail(ctx, FTK_EINVAL, "filter solves take one right-hand side");
        const int h = n_rhs / 2;
        CocgReq a = rq, b = rq;
        a.n_rhs = h;
        b.n_rhs = n_rhs - h;
        b.slots = rq.slots + h;
        if (rq.proj) b.proj = rq.proj + h;
        ftk_status s1 = cocg_core(ctx, a, G_out, iters_out, switches_out);
        if (s1 != FTK_OK && s1 != FTK_ENOCONV && s1 != FTK_EBREAKDOWN) return s1;
        ftk_status s2 = cocg_core(ctx, b, G_out + size_t(2) * h * n_omega, iters_out ? iters_out + h : nullptr,
                                  switches_out ? switches_out + h : nullptr);
        if (s2 != FTK_OK && s2 != FTK_ENOCONV && s2 != FTK_EBREAKDOWN) return s2;
        return s1 != FTK_OK ? s1 : s2;
    }
    ftk_status s;
    Plan *pl = nullptr;
    if ((s = get_plan(ctx, ctx->mprec, B, &pl))) return s;
    Small *d = ctx->dsmall;
    // per-RHS seed scalars: z_s = E_j + shift[seed]
    std::vector<double> e(n_rhs);
    for (int j = 0; j < n_rhs; ++j)
        CK(cudaMemcpyAsync(&e[j], ctx->slot_energy + rq.slots[j], sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const int mid = rq.seed_index >= 0 ? rq.seed_index : n_omega / 2;
    std::vector<CocgSeed> seeds(B);
    for (int j = 0; j < B; ++j) {
        memset(&seeds[j], 0, sizeof(CocgSeed));
        const int jj = j < n_rhs ? j : 0;          // padding lanes repeat RHS 0
        seeds[j].e0 = e[jj];
        seeds[j].zs_re = e[jj] + rq.shift[2 * mid];
        seeds[j].zs_im = rq.shift[2 * mid + 1];
        seeds[j].alpha_re = 1.0;
        seeds[j].seed_idx = mid;
    }
    CK(cudaMemcpyAsync(d->seed, seeds.data(), sizeof(CocgSeed) * B, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemsetAsync(d->inv_pi_max, 0, sizeof(d->inv_pi_max), ctx->stream));
    CK(cudaMemsetAsync(&d->all_done, 0, sizeof(int) * 2, ctx->stream));   // all_done, lowp
    dcx *om = (dcx *)wsp(ctx, ctx->L.omega);
    CK(cudaMemcpyAsync(om, rq.shift, sizeof(dcx) * n_omega, cudaMemcpyHostToDevice, ctx->stream));
    // shift arrays: pi_prev = pi_cur = 1, p~ = 0, G = 0
    const size_t sa_elems = size_t(B) * n_omega;
    dcx *sbase = (dcx *)wsp(ctx, ctx->L.shift);
    dcx *pi_prev = sbase, *pi_cur = sbase + sa_elems, *ptil = sbase + 2 * sa_elems, *G = sbase + 3 * sa_elems;
    {
        std::vector<double> ones(2 * sa_elems, 0.0);
        for (size_t i = 0; i < sa_elems; ++i) ones[2 * i] = 1.0;
        CK(cudaMemcpyAsync(pi_prev, ones.data(), sa_elems * 16, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(pi_cur, ones.data(), sa_elems * 16, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemsetAsync(ptil, 0, sa_elems * 16 * 3, ctx->stream));   // p~, G, frozen
        CK(cudaStreamSynchronize(ctx->stream));
    }
    void *kr[3] = {wsp(ctx, ctx->L.kry[0]), wsp(ctx, ctx->L.kry[1]), wsp(ctx, ctx->L.kry[2])};
    void *rcur = kr[0], *rprev = kr[1], *w = kr[2];

    UpdArgs ua{};
    ua.dim = ctx->dim;
    for (int j = 0; j < B; ++j) {
        const int jj = j < n_rhs ? j : 0;
        ua.lambda[j] = wsp(ctx, ctx->L.probes + ctx->L.vec_bytes * rq.slots[jj]);
        ua.proj[j] = rq.proj ? wsp(ctx, ctx->L.probes + ctx->L.vec_bytes * rq.proj[jj]) : nullptr;
    }
    ua.seed = d->seed;
    ua.partials = (double *)wsp(ctx, ctx->L.partials);
    ua.counter = &d->counters[3];
    ua.result = d->upd_dots;
    ua.all_done = &d->all_done;
    ua.lo_stride = (long long)ctx->max_rhs * (long long)ctx->dim;   // mixed and double-float modes
    ua.w_lo = ctx->prec == FTK_DF ? ua.lo_stride : 0;
    ua.lam_split = reinterpret_cast<float4 *>(wsp(ctx, ctx->L.lam_split));
    EpiArgs ea{};
    ea.partials = (double *)wsp(ctx, ctx->L.partials);
    ea.counter = &d->counters[4];
    ea.result = d->hv_dots;
    ea.all_done = &d->all_done;
    SeedArgs sa{};
    sa.n_rhs = B;
    sa.max_iter = rq.max_iter;
    sa.tol = rq.tol;
    sa.seed = d->seed;
    sa.upd = d->upd_dots;
    sa.hv = d->hv_dots;
    sa.inv_pi_max = d->inv_pi_max;
    sa.all_done = &d->all_done;
    sa.relax = ctx->relax;
    sa.lowp = &d->lowp;
    sa.seed_switch = rq.seed_switch;
    sa.n_omega = n_omega;
    sa.shift = om;
    sa.pi_prev = pi_prev;
    sa.pi_cur = pi_cur;
    ShiftArgs sh{};
    sh.n_omega = n_omega;
    sh.shift = om;
    sh.seed = d->seed;
    sh.pi_prev = pi_prev; sh.pi_cur = pi_cur; sh.ptil = ptil; sh.G = G;
    sh.inv_pi_max = d->inv_pi_max;
    sh.frozen = reinterpret_cast<int *>(sbase + 4 * sa_elems);
    sh.tol = rq.tol;
    sh.hist = rq.hist;
    sh.hist_cap = rq.hist_cap;
    sa.frozen = sh.frozen;
    SwitchArgs swa{};
    swa.kind = upd_kind(ctx);
    swa.dim = ctx->dim;
    swa.lo_stride = ua.lo_stride;
    swa.w_lo = ctx->prec == FTK_DF ? ua.lo_stride : 0;
    swa.seed = d->seed;
    swa.pi_prev = pi_prev;
    swa.pi_cur = pi_cur;
    swa.n_omega = n_omega;
    swa.all_done = &d->all_done;
    IterExtras ex{rq.seed_switch ? &swa : nullptr, rq.acc};

    // r_0 = lambda (+ dots); r_{-1} = 0 so that c_0 r_{-1} is exactly zero
    if (ctx->prec >= FTK_MIXED) {   // hi and lo parts of the B columns
        CK(cudaMemsetAsync(rprev, 0, ctx->dim * 8 * B, ctx->stream));
        CK(cudaMemsetAsync(static_cast<char *>(rprev) + size_t(8) * ua.lo_stride, 0, ctx->dim * 8 * B, ctx->stream));
    } else {
        CK(cudaMemsetAsync(rprev, 0, ctx->L.vec_bytes * B, ctx->stream));
    }
    ua.mode = 0;
    LAUNCH(launch_cocg_update(upd_kind(ctx), B, nullptr, nullptr, rcur, ua, vec_grid(ctx, ctx->dim), ctx->stream));
    int it0 = 0;
    if (ctx->prec == FTK_DF) {
        // step 0 without the fused update: W = H r_0 (+mu), seed, shifts
        EpiArgs e0 = ea;
        e0.df_lo = ua.lo_stride;
        if ((s = run_hv(ctx, ctx->mprec, B, EPI_COCG, rcur, w, e0))) return s;
        LAUNCH(launch_cocg_seed(sa, ctx->stream));
        LAUNCH(launch_cocg_shift(sh, B, ctx->stream));
        it0 = 1;
    }

    // Capture two iterations (buffer roles return to the start) in a graph.
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const int64_t l0 = ctx->launches;
    int64_t per_graph = 0;
    cudaError_t ce = cudaSuccess;
    {
        std::lock_guard<std::mutex> lk(device_mu());
        CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        ftk_status cs = cocg_iteration(ctx, B, rcur, rprev, w, ea, sa, sh, ua, ex);
        if (cs == FTK_OK) cs = cocg_iteration(ctx, B, rprev, rcur, w, ea, sa, sh, ua, ex);
        ce = cudaStreamEndCapture(ctx->stream, &graph);
        if (cs != FTK_OK) { if (graph) cudaGraphDestroy(graph); return cs; }
        CK(ce);
        per_graph = ctx->launches - l0;
        ctx->launches = l0;
        const ftk_status is = instantiate_cached(ctx, graph, &exec);
        cudaGraphDestroy(graph);
        if (is != FTK_OK) return is;
    }
    int done = 0, it = it0;
    const int chunk = 16;   // graph launches between host checks (32 iterations)
    ftk_status result = FTK_OK;
    while (!done) {
        for (int g = 0; g < chunk && it <= rq.max_iter + 2; ++g, it += 2) {
            ce = cudaGraphLaunch(exec, ctx->stream);
            if (ce != cudaSuccess) break;
            ctx->launches += per_graph;
        }
        if (ce != cudaSuccess) break;
        ce = cudaMemcpyAsync(&done, &d->all_done, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->stream);
        if (ce != cudaSuccess) break;
        if (it > rq.max_iter + 2) break;
    }
    CK(ce);
    // results
    std::vector<CocgSeed> out(B);
    CK(cudaMemcpyAsync(out.data(), d->seed, sizeof(CocgSeed) * B, cudaMemcpyDeviceToHost, ctx->stream));
    std::vector<double> g(2 * sa_elems);
    CK(cudaMemcpyAsync(g.data(), G, sa_elems * 16, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    std::string why;
    for (int j = 0; j < n_rhs; ++j) {
        if (G_out) memcpy(G_out + size_t(2) * j * n_omega, g.data() + size_t(2) * j * n_omega, sizeof(double) * 2 * n_omega);
        if (iters_out) iters_out[j] = out[j].iters;
        if (switches_out) switches_out[j] = out[j].switches;
        const int dn = out[j].done;
        if ((dn == 2 || dn == 3 || dn == 5) && result != FTK_EBREAKDOWN) {
            result = FTK_EBREAKDOWN;
            why = "shifted COCG breakdown (rhs " + std::to_string(j) + ", iteration " + std::to_string(out[j].iters) +
                  ", " + (dn == 2 ? "r^T r vanished" : dn == 3 ? "alpha denominator vanished" : "non-finite residual") +
                  ")";
        }
        if ((dn == 4 || dn == 0) && result == FTK_OK) result = FTK_ENOCONV;
    }
    if (result == FTK_ENOCONV) ctx->err = "shifted COCG reached max_iter";
    if (result == FTK_EBREAKDOWN) ctx->err = why;
    return result;
}

static ftk_status check_cocg_args(ftk_ctx *ctx, const int32_t *slots, const int32_t *proj, int32_t n_rhs,
                                  int32_t n_shift, double tol, int32_t max_iter) {
    if (!slots || n_rhs < 1 || n_rhs > FTK_MAX_RHS * 64 || n_shift < 1 || n_shift > FTK_MAX_OMEGA || !(tol > 0) ||
        max_iter < 1)
        return fail(ctx, FTK_EINVAL, "bad shifted COCG arguments");
    for (int j = 0; j < n_rhs; ++j) {
        if (slots[j] < 0 || slots[j] >= ctx->max_rhs || !ctx->slot_valid[slots[j]])
            return fail(ctx, FTK_EINVAL, "rhs slot not loaded");
        if (proj && (proj[j] < 0 || proj[j] >= ctx->max_rhs || !ctx->slot_valid[proj[j]]))
            return fail(ctx, FTK_EINVAL, "projection slot not loaded");
    }
    return FTK_OK;
}

ftk_status ftk_shifted_cocg(ftk_ctx *ctx, const int32_t *slots, int32_t n_rhs, const double *omega,
                            int32_t n_omega, double eta, double tol, int32_t max_iter, double *G_out,
                            int32_t *iters_out) {
    ftk_status s = check_ready(ctx);
    if (s) return s;
    if (!omega || !G_out || !(eta > 0) || n_rhs > ctx->max_rhs)
        return fail(ctx, FTK_EINVAL, "bad shifted COCG arguments");
    if ((s = check_cocg_args(ctx, slots, nullptr, n_rhs, n_omega, tol, max_iter))) return s;
    std::vector<double> z(2 * size_t(n_omega));
    for (int i = 0; i < n_omega; ++i) { z[2 * i] = omega[i]; z[2 * i + 1] = eta; }
    CocgReq rq;
    rq.slots = slots;
    rq.n_rhs = n_rhs;
    rq.shift = z.data();
    rq.n_shift = n_omega;
    rq.tol = tol;
    rq.max_iter = max_iter;
    return cocg_core(ctx, rq, G_out, iters_out, nullptr);
}

ftk_status ftk_shifted_cocg_ex(ftk_ctx *ctx, const int32_t *rhs_slots, int32_t n_rhs, const double *shifts,
                               int32_t n_shift, double tol, int32_t max_iter, const ftk_cocg_opts *opts,
                               double *G_out, int32_t *iters_out, int32_t *switches_out) {
    ftk_status s = check_ready(ctx);
    if (s) return s;
    const int32_t *proj = opts ? opts->proj_slots : nullptr;
    if (!shifts || !G_out || n_rhs > ctx->max_rhs) return fail(ctx, FTK_EINVAL, "bad shifted COCG arguments");
    if ((s = check_cocg_args(ctx, rhs_slots, proj, n_rhs, n_shift, tol, max_iter))) return s;
    for (int i = 0; i < n_shift; ++i)
        if (!std::isfinite(shifts[2 * i]) || !(shifts[2 * i + 1] > 0))
            return fail(ctx, FTK_EINVAL, "shifts must be finite with positive imaginary part");
    CocgReq rq;
    rq.slots = rhs_slots;
    rq.proj = proj;
    rq.n_rhs = n_rhs;
    rq.shift = shifts;
    rq.n_shift = n_shift;
    rq.tol = tol;
    rq.max_iter = max_iter;
    if (opts) {
        if (opts->seed_index < -1 || opts->seed_index >= n_shift)
            return fail(ctx, FTK_EINVAL, "seed_index out of range");
        rq.seed_index = opts->seed_index;
        rq.seed_switch = opts->seed_switch ? 1 : 0;
    }
    return cocg_core(ctx, rq, G_out, iters_out, switches_out);
}

// ---------------------------------------------------------------- cTPQ (f2)
// Appendix A: exp(N b (l - h)/2) psi applied as M_d Taylor steps of
// tau = N db / (2 M_d) for each increment db of the (ascending) beta list.
// The step count comes from the fixed point of X_{j+1} = ln Lambda + ln(2 pi X_j)/2
// (the largest term X^k/k! of a step is then about Lambda), X_0 = Lambda,
// M_d = ceil(N db (l + |eps_0|) / (2 X)). |eps_0| is bounded by the bond
// spectrum: (1/N) sum_b |lambda_min(h_b)|. One step sums
// t_0 = v, t_{k+1} = tau/(k+1) (l - h) t_k up to the first k >= X with
// X^k / k! <= 1e-17: since l - h is positive semidefinite the sum is at least
// |v|, and |t_k| <= X^k/k! |v|, so the dropped tail is below 1e-17 of it.
static int ctpq_steps(int n, double dbeta, double ell, double eps0, double lam, double *x_out) {
    double x = lam;
    for (int i = 0; i < 1000; ++i) {
        const double nx = std::log(lam) + 0.5 * std::log(2.0 * M_PI * x);
        const bool fin = std::fabs(nx - x) <= 1e-15 * std::fabs(nx);
        x = nx;
        if (fin) break;
    }
    *x_out = x;
    const double md = std::ceil(n * dbeta / 2.0 * (ell + eps0) / x);
    return std::max(1, (int)md);
}

static int taylor_terms(double X) {
    int k = 1;
    while (k < 100000) {
        if (k >= X && k * std::log(std::max(X, 1e-300)) - std::lgamma(k + 1.0) <= std::log(1e-17)) break;
        ++k;
    }
    return k;
}

ftk_status ftk_ctpq(ftk_ctx *ctx, const double *beta, int32_t n_beta, double lam, int32_t first_shell,
                    double *log_norm_out, int32_t *md_out, double *energy_out) {
    ftk_status s = check_ready(ctx);
    if (s) return s;
    if (!ctx->have_state) return fail(ctx, FTK_EBUSY, "no TPQ state: call ftk_tpq_init first");
    if (!beta || n_beta < 1 || !(lam > 1.0) || first_shell < 0 || first_shell + n_beta > ctx->n_saved_cap)
        return fail(ctx, FTK_EINVAL, "ftk_ctpq: bad arguments (beta list, Lambda > 1, shells within n_saved)");
    for (int i = 0; i < n_beta; ++i)
        if (!(beta[i] >= 0.0) || !std::isfinite(beta[i]) || (i > 0 && beta[i] < beta[i - 1]))
            return fail(ctx, FTK_EINVAL, "ftk_ctpq: betas must be finite, >= 0 and ascending");
    if (ctx->L.vec_bytes * 3 * (size_t)ctx->max_rhs < ctx->dim * 32)
        return fail(ctx, FTK_ENOMEM, "ftk_ctpq: the Krylov region must hold two FP64 vectors");
    Plan *pl64 = nullptr;
    if ((s = get_plan(ctx, FTK_FP64, 1, &pl64))) return s;
    const double lmin = std::min({(ctx->J + ctx->K) / 4, (ctx->J - ctx->K) / 4, -(3 * ctx->J + ctx->K) / 4});
    const double eps0 = ctx->nb * std::fabs(lmin) / ctx->n;
    // buffers: V = psi[0] (the state), C = psi[1] (the step's sum), terms in the Krylov region
    double2 *V = (double2 *)wsp(ctx, ctx->L.psi[0]);
    double2 *C = (double2 *)wsp(ctx, ctx->L.psi[1]);
    double2 *T0 = (double2 *)wsp(ctx, ctx->L.kry[0]);
    double2 *T1 = T0 + ctx->dim;
    double *dscale = &ctx->dsmall->op_dots[3];
    // the current state, normalised, into V (through T0 when it already is V)
    const void *cur = wsp(ctx, ctx->L.psi[ctx->k & 1]);
    LAUNCH(launch_convert_out(FTK_FP64, cur, T0, ctx->dim, &ctx->dsmall->tpq.scale, vec_grid(ctx, ctx->dim),
                              ctx->stream));
    CK(cudaMemcpyAsync(V, T0, ctx->dim * 16, cudaMemcpyDeviceToDevice, ctx->stream));
    EpiArgs ea{};
    ea.ell = ctx->ell;
    ea.inv_n = 1.0 / ctx->n;
    ea.partials = (double *)wsp(ctx, ctx->L.partials);
    ea.counter = &ctx->dsmall->counters[1];
    ea.result = ctx->dsmall->op_dots;
    ea.taylor_acc = C;
    double log_norm = 0.0, prev = 0.0;
    for (int i = 0; i < n_beta; ++i) {
        const double db = beta[i] - prev;
        prev = beta[i];
        int md = 0;
        if (db > 0.0) {
            double X = 0;
            md = ctpq_steps(ctx->n, db, ctx->ell, eps0, lam, &X);
            const double tau = ctx->n * db / (2.0 * md);
            const int kmax = taylor_terms(tau * (ctx->ell + eps0));
            for (int st = 0; st < md; ++st) {
                CK(cudaMemcpyAsync(C, V, ctx->dim * 16, cudaMemcpyDeviceToDevice, ctx->stream));
                const double2 *in = V;
                for (int k = 0; k < kmax; ++k) {
                    double2 *out = (k & 1) ? T1 : T0;
                    EpiArgs e = ea;
                    e.tcoef = tau / (k + 1);
                    if ((s = run_hv(ctx, FTK_FP64, 1, EPI_TAYLOR, in, out, e))) return s;
                    in = out;
                }
                // V = C / |C|, log |C| accumulated
                double n2 = 0;
                CK(cudaMemcpyAsync(&n2, ctx->dsmall->op_dots + 1, sizeof n2, cudaMemcpyDeviceToHost, ctx->stream));
                CK(cudaStreamSynchronize(ctx->stream));
                if (!(n2 > 0) || !std::isfinite(n2)) return fail(ctx, FTK_EBREAKDOWN, "ftk_ctpq: non-finite Taylor sum");
                log_norm += 0.5 * std::log(n2);
                const double sc = 1.0 / std::sqrt(n2);
                CK(cudaMemcpyAsync(dscale, &sc, sizeof sc, cudaMemcpyHostToDevice, ctx->stream));
                LAUNCH(launch_convert_out(FTK_FP64, C, V, ctx->dim, dscale, vec_grid(ctx, ctx->dim), ctx->stream));
            }
        }
        // energy <phi|H|phi> of the normalised state: one Taylor pass with c = 0
        CK(cudaMemcpyAsync(C, V, ctx->dim * 16, cudaMemcpyDeviceToDevice, ctx->stream));
        EpiArgs e = ea;
        e.tcoef = 0.0;
        if ((s = run_hv(ctx, FTK_FP64, 1, EPI_TAYLOR, V, T0, e))) return s;
        double en = 0;
        CK(cudaMemcpyAsync(&en, ctx->dsmall->op_dots, sizeof en, cudaMemcpyDeviceToHost, ctx->stream));
        // the state into its shell (context vector precision), scale 1, origin its energy
        const int sidx = first_shell + i;
        void *dst = wsp(ctx, ctx->L.shells + ctx->L.vec_bytes * sidx);
        if (ctx->vprec == 0)
            CK(cudaMemcpyAsync(dst, V, ctx->L.vec_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
        else
            LAUNCH(launch_convert_in(ctx->vprec, V, dst, ctx->dim, vec_grid(ctx, ctx->dim), ctx->stream));
        const double one = 1.0;
        CK(cudaMemcpyAsync(ctx->shell_scale + sidx, &one, sizeof one, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        if ((int)ctx->shell_step.size() <= sidx) {
            ctx->shell_step.resize(sidx + 1, -1);
            ctx->shell_origin.resize(sidx + 1, NAN);
        }
        ctx->shell_step[sidx] = -1;
        ctx->shell_origin[sidx] = en;
        ctx->n_saved = std::max(ctx->n_saved, sidx + 1);
        if (log_norm_out) log_norm_out[i] = log_norm;
        if (md_out) md_out[i] = md;
        if (energy_out) energy_out[i] = en;
    }
    // the TPQ state becomes the last cTPQ state (normalised, step counter 0)
    TpqState h{};
    h.scale = 1.0;
    h.ell = ctx->ell;
    h.n_sites = ctx->n;
    CK(cudaMemcpyAsync(&ctx->dsmall->tpq, &h, sizeof h, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->k = 0;
    return FTK_OK;
}

// ------------------------------------------------------ filter shells (f1)
// Eq. dfilterP / Eq. filtered: phi^m = (1/M) sum_j rho e^{i th_j} (E_m + rho e^{i th_j} - H)^{-1} phi,
// th_j = 2 pi (j - 1/2) / M, E_m = E_b + (2m + 1) eps, rho = eps. All L M
// resolvents share the right-hand side phi, so ONE shifted COCG over the L M
// contour points serves every shell. The solution vectors are not kept per
// shift: pass 1 runs the solve and records the shift recurrences; from them
// x^s = sum_k C^s_k r_k (backward sums); pass 2 replays the same solve
// (deterministic reductions: the same r_k) and accumulates
// phi^m += sum_j w_j C^{(m, j)}_k r_k into L vectors.
static size_t filter_hist_bytes(int L, int M, int max_iter) { return align_up(size_t(48) * L * M * max_iter); }
static size_t filter_coef_bytes(int L, int max_iter) { return align_up(size_t(16) * L * max_iter); }

size_t ftk_filter_footprint(int32_t n_centres, int32_t n_points, int32_t max_iter) {
    if (n_centres < 1 || n_points < 1 || n_points > 32 || (size_t)n_centres * n_points > FTK_MAX_OMEGA ||
        max_iter < 1)
        return 0;
    return filter_hist_bytes(n_centres, n_points, max_iter) + filter_coef_bytes(n_centres, max_iter) +
           align_up(size_t(16) * n_points);
}

ftk_status ftk_filter_shells(ftk_ctx *ctx, int32_t src, double e_b, double eps, int32_t n_centres, int32_t n_points,
                             double tol, int32_t max_iter, void *scratch, size_t scratch_bytes, int32_t first_shell,
                             double *norm2_out, int32_t *iters_out) {
    ftk_status s = check_ready(ctx);
    if (s) return s;
    const int L = n_centres, M = n_points;
    if (ctx->prec != FTK_FP64) return fail(ctx, FTK_EINVAL, "ftk_filter_shells: needs precision FTK_FP64");
    const size_t need = ftk_filter_footprint(L, M, max_iter);
    if (need == 0 || !std::isfinite(e_b) || !(eps > 0) || !(tol > 0) || first_shell < 0 ||
        first_shell + L > ctx->n_saved_cap)
        return fail(ctx, FTK_EINVAL, "ftk_filter_shells: bad arguments (M <= 32, L M <= 4096, shells within n_saved)");
    if (!scratch || scratch_bytes < need || (reinterpret_cast<uintptr_t>(scratch) % kAlign))
        return fail(ctx, FTK_ENOMEM, "ftk_filter_shells: scratch missing, unaligned or smaller than ftk_filter_footprint");
    // source phi (normalised) into probe slot 0, shift origin 0
    const void *sv = nullptr;
    const double *scale = nullptr;
    if (src == 0) {
        if (!ctx->have_state) return fail(ctx, FTK_EBUSY, "no TPQ state");
        sv = wsp(ctx, ctx->L.psi[ctx->k & 1]);
        scale = &ctx->dsmall->tpq.scale;
    } else {
        const int sh = src - 1;
        if (!shell_written(ctx, sh)) return fail(ctx, FTK_EINVAL, "ftk_filter_shells: no such source shell");
        if (sh >= first_shell && sh < first_shell + L)
            return fail(ctx, FTK_EINVAL, "ftk_filter_shells: the source shell would be overwritten");
        sv = wsp(ctx, ctx->L.shells + ctx->L.vec_bytes * sh);
        scale = ctx->shell_scale + sh;
    }
    double2 *lam = (double2 *)wsp(ctx, ctx->L.probes);
    LAUNCH(launch_convert_out(FTK_FP64, sv, lam, ctx->dim, scale, vec_grid(ctx, ctx->dim), ctx->stream));
    const double zero = 0.0;
    CK(cudaMemcpyAsync(ctx->slot_energy, &zero, sizeof zero, cudaMemcpyHostToDevice, ctx->stream));
    ctx->slot_valid[0] = 1;
    // contour points z = E_m + eps e^{i th_j} (shift s = m M + j) and weights
    std::vector<double> z(2 * size_t(L) * M);
    std::vector<dcx> w(M);
    for (int j = 0; j < M; ++j) {
        const double th = 2.0 * M_PI * (j + 0.5) / M;
        w[j] = {eps * std::cos(th) / M, eps * std::sin(th) / M};
        for (int m = 0; m < L; ++m) {
            const double em = e_b + (2 * m + 1) * eps;
            z[2 * (size_t(m) * M + j)] = em + eps * std::cos(th);
            z[2 * (size_t(m) * M + j) + 1] = eps * std::sin(th);
        }
    }
    char *scr = static_cast<char *>(scratch);
    dcx *hist = reinterpret_cast<dcx *>(scr);
    dcx *coef = reinterpret_cast<dcx *>(scr + filter_hist_bytes(L, M, max_iter));
    dcx *wdev = reinterpret_cast<dcx *>(scr + filter_hist_bytes(L, M, max_iter) + filter_coef_bytes(L, max_iter));
    CK(cudaMemcpyAsync(wdev, w.data(), sizeof(dcx) * M, cudaMemcpyHostToDevice, ctx->stream));
    const int32_t slot0 = 0;
    CocgReq rq;
    rq.slots = &slot0;
    rq.n_rhs = 1;
    rq.shift = z.data();
    rq.n_shift = L * M;
    rq.seed_index = (L / 2) * M;   // th = pi / M: the smallest positive imaginary part
    rq.tol = tol;
    rq.max_iter = max_iter;
    rq.hist = hist;
    rq.hist_cap = max_iter;
    int32_t it1 = 0, it2 = 0;
    s = cocg_core(ctx, rq, nullptr, &it1, nullptr);
    if (s != FTK_OK) return s;
    FilterCoefArgs fc{};
    fc.n_iter = it1;
    fc.L = L;
    fc.M = M;
    fc.hist = hist;
    fc.w = wdev;
    fc.coef = coef;
    LAUNCH(launch_filter_coef(fc, ctx->stream));
    double2 *phi = (double2 *)wsp(ctx, ctx->L.shells + ctx->L.vec_bytes * first_shell);
    CK(cudaMemsetAsync(phi, 0, ctx->L.vec_bytes * L, ctx->stream));
    FilterAccArgs fa{};
    fa.dim = ctx->dim;
    fa.L = L;
    fa.n_coef = it1;
    fa.phi = phi;
    fa.coef = coef;
    fa.seed = ctx->dsmall->seed;
    rq.hist = nullptr;
    rq.hist_cap = 0;
    rq.acc = &fa;
    s = cocg_core(ctx, rq, nullptr, &it2, nullptr);
    if (s != FTK_OK) return s;
    if (it2 != it1) return fail(ctx, FTK_ECUDA, "ftk_filter_shells: the second pass did not replay the first");
    // norms <phi^m|phi^m>, shell metadata (scale 1, origin E_m)
    std::vector<double> one(L, 1.0);
    CK(cudaMemcpyAsync(ctx->shell_scale + first_shell, one.data(), sizeof(double) * L, cudaMemcpyHostToDevice,
                       ctx->stream));
    if ((int)ctx->shell_step.size() < first_shell + L) {
        ctx->shell_step.resize(first_shell + L, -1);
        ctx->shell_origin.resize(first_shell + L, NAN);
    }
    for (int m = 0; m < L; ++m) {
        InitArgs ia{};
        ia.dim = ctx->dim;
        ia.partials = (double *)wsp(ctx, ctx->L.partials);
        ia.counter = &ctx->dsmall->counters[0];
        ia.result = ctx->dsmall->op_dots + 2;
        LAUNCH(launch_norm(FTK_FP64, phi + size_t(m) * ctx->dim, ia, vec_grid(ctx, ctx->dim), ctx->stream));
        double n2 = 0;
        CK(cudaMemcpyAsync(&n2, ctx->dsmall->op_dots + 2, sizeof n2, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        if (norm2_out) norm2_out[m] = n2;
        ctx->shell_step[first_shell + m] = -1;
        ctx->shell_origin[first_shell + m] = e_b + (2 * m + 1) * eps;
    }
    ctx->n_saved = std::max(ctx->n_saved, first_shell + L);
    if (iters_out) *iters_out = it1;
    return FTK_OK;
}

ftk_status ftk_filter_spectrum(ftk_ctx *ctx, const double *Gh, int32_t n_shell, int32_t n_omega, const double *energy,
                               const double *norm2, double beta, double eps, const double *T, int32_t n_T,
                               double *S_out, double *P_out) {
    ftk_status s = check_ready(ctx);
    if (s) return s;
    if (!Gh || !energy || !norm2 || !T || !S_out || n_shell < 1 || n_shell > 1024 || n_omega < 1 ||
        n_omega > FTK_MAX_OMEGA || n_T < 1 || n_T > 1024 || !std::isfinite(beta) || !(eps > 0))
        return fail(ctx, FTK_EINVAL, "bad filter spectrum arguments");
    for (int t = 0; t < n_T; ++t)
        if (!(T[t] > 0)) return fail(ctx, FTK_EINVAL, "temperatures must be positive");
    for (int q = 0; q < n_shell; ++q)
        if (!std::isfinite(energy[q]) || !(norm2[q] >= 0)) return fail(ctx, FTK_EINVAL, "bad shell energy or norm");
    double *gb = (double *)wsp(ctx, ctx->L.gbuf);
    double *tb = (double *)wsp(ctx, ctx->L.tbuf);
    double *eb = tb + 1024, *nb = tb + 2048;
    const size_t s_need = size_t(n_T) * n_omega * 8 + size_t(n_T) * n_shell * 8 + 16;
    const size_t g_used = align_up(size_t(16) * n_shell * n_omega);
    double *sb = (double *)wsp(ctx, ctx->L.kry[0]);
    if (ctx->L.vec_bytes * ctx->max_rhs < s_need) {
        if (g_used + s_need > ctx->L.tbuf - ctx->L.gbuf)
            return fail(ctx, FTK_ENOMEM, "no workspace region large enough to stage the spectrum");
        sb = (double *)wsp(ctx, ctx->L.gbuf + g_used);
    }
    double *pb = sb + size_t(n_T) * n_omega;
    CK(cudaMemcpyAsync(gb, Gh, size_t(16) * n_shell * n_omega, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(tb, T, sizeof(double) * n_T, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(eb, energy, sizeof(double) * n_shell, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(nb, norm2, sizeof(double) * n_shell, cudaMemcpyHostToDevice, ctx->stream));
    FrwArgs fa{};
    fa.n_shell = n_shell;
    fa.n_omega = n_omega;
    fa.beta = beta;
    fa.eps = eps;
    fa.E = eb;
    fa.norm2 = nb;
    fa.G = gb;
    fa.T = tb;
    fa.S = sb;
    fa.P = pb;
    LAUNCH(launch_frw_spectrum(fa, n_T, ctx->stream));
    CK(cudaMemcpyAsync(S_out, sb, sizeof(double) * n_T * n_omega, cudaMemcpyDeviceToHost, ctx->stream));
    if (P_out) CK(cudaMemcpyAsync(P_out, pb, sizeof(double) * n_T * n_shell, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return FTK_OK;
}

ftk_status ftk_spectrum(ftk_ctx *ctx, const double *Gh, int32_t n_shell, int32_t n_omega, const double *T,
                        int32_t n_T, double *S_out, int32_t *trunc_out) {
    ftk_status s = check_ready(ctx);
    if (s) return s;
    if (!Gh || !T || !S_out || n_shell < 1 || n_shell > ctx->n_saved || n_shell > 1024 || n_omega < 1 ||
        n_omega > FTK_MAX_OMEGA || n_T < 1 || n_T > 1024)
        return fail(ctx, FTK_EINVAL, "bad spectrum arguments");
    for (int t = 0; t < n_T; ++t)
        if (!(T[t] > 0)) return fail(ctx, FTK_EINVAL, "temperatures must be positive");
    // the reweighting reads the mTPQ statistics of every step k < ctx->k: the
    // shells must be the mTPQ shells 0 .. n_shell-1 of the current sequence
    if (ctx->k < 1 || !ctx->stats) return fail(ctx, FTK_EBUSY, "no mTPQ statistics: run ftk_tpq_step first");
    for (int q = 0; q < n_shell; ++q)
        if (ctx->shell_step[q] != q * ctx->save_every)
            return fail(ctx, FTK_EINVAL, "ftk_spectrum reweights mTPQ shells (use ftk_filter_spectrum for filtered ones)");
    double *gb = (double *)wsp(ctx, ctx->L.gbuf);
    double *tb = (double *)wsp(ctx, ctx->L.tbuf);
    // S and trunc are staged in the Krylov region or, for small clusters,
    // behind the G input in its staging region
    const size_t s_need = size_t(n_T) * n_omega * 8 + n_T * 4 + 16;
    const size_t g_used = align_up(size_t(16) * n_shell * n_omega);
    double *sb = (double *)wsp(ctx, ctx->L.kry[0]);
    if (ctx->L.vec_bytes * ctx->max_rhs < s_need) {
        if (g_used + s_need > ctx->L.tbuf - ctx->L.gbuf)
            return fail(ctx, FTK_ENOMEM, "no workspace region large enough to stage the spectrum");
        sb = (double *)wsp(ctx, ctx->L.gbuf + g_used);
    }
    int *trb = (int *)(sb + size_t(n_T) * n_omega);
    CK(cudaMemcpyAsync(gb, Gh, size_t(16) * n_shell * n_omega, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(tb, T, sizeof(double) * n_T, cudaMemcpyHostToDevice, ctx->stream));
    SpecArgs sp{};
    sp.n_sites_i = ctx->n;
    sp.n_sites = ctx->n;
    sp.ell = ctx->ell;
    sp.n_steps = ctx->k;
    sp.save_every = ctx->save_every;
    sp.n_shell = n_shell;
    sp.n_omega = n_omega;
    sp.u = stat_u(ctx);
    sp.logq = stat_lq(ctx);
    sp.G = gb;
    sp.T = tb;
    sp.S = sb;
    sp.trunc = trb;
    LAUNCH(launch_spectrum(sp, n_T, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpyAsync(S_out, sb, sizeof(double) * n_T * n_omega, cudaMemcpyDeviceToHost, ctx->stream));
    std::vector<int> tr(n_T);
    CK(cudaMemcpyAsync(tr.data(), trb, sizeof(int) * n_T, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    int any = 0;
    for (int t = 0; t < n_T; ++t) {
        if (trunc_out) trunc_out[t] = tr[t];
        any |= tr[t];
    }
    return any ? FTK_ETRUNC : FTK_OK;
}

ftk_status ftk_spectrum_ex(ftk_ctx *ctx, const double *Gh, int32_t n_shell, int32_t n_omega, const double *T,
                           int32_t n_T, const double *u, const double *logQ, int32_t n_steps, int32_t save_every,
                           double ell, double *S_out, int32_t *trunc_out) {
    ftk_status s = check_ready(ctx);
    if (s) return s;
    if (!Gh || !T || !S_out || !u || !logQ || n_shell < 1 || n_shell > 1024 || n_omega < 1 ||
        n_omega > FTK_MAX_OMEGA || n_T < 1 || n_T > 1024 || n_steps < 1 || save_every < 1 ||
        (size_t)n_steps * 16 > kPartialsBytes || (n_shell - 1) * save_every >= n_steps || !std::isfinite(ell))
        return fail(ctx, FTK_EINVAL, "bad spectrum arguments");
    for (int t = 0; t < n_T; ++t)
        if (!(T[t] > 0)) return fail(ctx, FTK_EINVAL, "temperatures must be positive");
    for (int k = 0; k < n_steps; ++k)
        if (!(ell - u[k] > 0) || !std::isfinite(logQ[k])) return fail(ctx, FTK_EINVAL, "need l > u_k and finite log Q_k");
    double *gb = (double *)wsp(ctx, ctx->L.gbuf);
    double *tb = (double *)wsp(ctx, ctx->L.tbuf);
    double *ub = (double *)wsp(ctx, ctx->L.partials), *qb = ub + n_steps;
    const size_t s_need = size_t(n_T) * n_omega * 8 + n_T * 4 + 16;
    const size_t g_used = align_up(size_t(16) * n_shell * n_omega);
    double *sb = (double *)wsp(ctx, ctx->L.kry[0]);
    if (ctx->L.vec_bytes * ctx->max_rhs < s_need) {
        if (g_used + s_need > ctx->L.tbuf - ctx->L.gbuf)
            return fail(ctx, FTK_ENOMEM, "no workspace region large enough to stage the spectrum");
        sb = (double *)wsp(ctx, ctx->L.gbuf + g_used);
    }
    int *trb = (int *)(sb + size_t(n_T) * n_omega);
    CK(cudaMemcpyAsync(gb, Gh, size_t(16) * n_shell * n_omega, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(tb, T, sizeof(double) * n_T, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ub, u, sizeof(double) * n_steps, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(qb, logQ, sizeof(double) * n_steps, cudaMemcpyHostToDevice, ctx->stream));
    SpecArgs sp{};
    sp.n_sites_i = ctx->n;
    sp.n_sites = ctx->n;
    sp.ell = ell;
    sp.n_steps = n_steps;
    sp.save_every = save_every;
    sp.n_shell = n_shell;
    sp.n_omega = n_omega;
    sp.u = ub;
    sp.logq = qb;
    sp.G = gb;
    sp.T = tb;
    sp.S = sb;
    sp.trunc = trb;
    LAUNCH(launch_spectrum(sp, n_T, ctx->stream));
    CK(cudaMemcpyAsync(S_out, sb, sizeof(double) * n_T * n_omega, cudaMemcpyDeviceToHost, ctx->stream));
    std::vector<int> tr(n_T);
    CK(cudaMemcpyAsync(tr.data(), trb, sizeof(int) * n_T, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    int any = 0;
    for (int t = 0; t < n_T; ++t) {
        if (trunc_out) trunc_out[t] = tr[t];
        any |= tr[t];
    }
    return any ? FTK_ETRUNC : FTK_OK;
}

ftk_status ftk_hv(ftk_ctx *ctx, const void *v_dev, void *out_dev, int32_t n_rhs) {
    if (!ctx) return FTK_EINVAL;
    if (!v_dev || !out_dev || v_dev == out_dev) return fail(ctx, FTK_EINVAL, "bad vectors");
    if ((reinterpret_cast<uintptr_t>(v_dev) | reinterpret_cast<uintptr_t>(out_dev)) & 15)
        return fail(ctx, FTK_EINVAL, "vectors must be 16-byte aligned");
    if (n_rhs < 1 || n_rhs > FTK_MAX_RHS || (n_rhs & (n_rhs - 1)))
        return fail(ctx, FTK_EINVAL, "n_rhs must be a power of two <= 32");
    EpiArgs ea{};
    if (ctx->mprec == 2) ea.df_lo = (long long)n_rhs * (long long)ctx->dim;   // hi block, then lo block
    return run_hv(ctx, ctx->mprec, n_rhs, EPI_PLAIN, v_dev, out_dev, ea);
}

ftk_status ftk_get_vector(ftk_ctx *ctx, int32_t which, double *host_out) {
    ftk_status s = check_ready(ctx);
    if (s) return s;
    if (!host_out) return fail(ctx, FTK_EINVAL, "null output");
    const void *src = nullptr;
    const double *scale = nullptr;
    if (which == 0) {
        if (!ctx->have_state) return fail(ctx, FTK_EBUSY, "no TPQ state");
        src = wsp(ctx, ctx->L.psi[ctx->k & 1]);
        scale = &ctx->dsmall->tpq.scale;
    } else if (which > 0) {
        const int sh = which - 1;
        if (!shell_written(ctx, sh)) return fail(ctx, FTK_EINVAL, "no such shell");
        src = wsp(ctx, ctx->L.shells + ctx->L.vec_bytes * sh);
        scale = ctx->shell_scale + sh;
    } else {
        const int sl = -1 - which;
        if (sl >= ctx->max_rhs || !ctx->slot_valid[sl]) return fail(ctx, FTK_EINVAL, "no such probe");
        src = wsp(ctx, ctx->L.probes + ctx->L.vec_bytes * sl);
    }
    void *stage = wsp(ctx, ctx->L.kry[0]);
    LAUNCH(launch_convert_out(which == 0 ? FTK_FP64 : ctx->vprec, src, stage, ctx->dim, scale,
                              vec_grid(ctx, ctx->dim), ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpyAsync(host_out, stage, ctx->dim * 16, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return FTK_OK;
}

ftk_status ftk_plan_info(const ftk_ctx *cctx, int32_t *n_passes, int32_t *tile_bits) {
    ftk_ctx *ctx = const_cast<ftk_ctx *>(cctx);
    if (!ctx) return FTK_EINVAL;
    Plan *pl = nullptr;
    ftk_status s = get_plan(ctx, ctx->mprec, 1, &pl);
    if (s) return s;
    if (n_passes) *n_passes = (int)pl->passes.size();
    if (tile_bits) *tile_bits = pl->tile_bits;
    return FTK_OK;
}

ftk_status ftk_set_relax(ftk_ctx *ctx, double theta) {
    if (!ctx) return fail(nullptr, FTK_EINVAL, "null context");
    if (!(theta >= 0.0) || !std::isfinite(theta)) return fail(ctx, FTK_EINVAL, "theta must be finite and >= 0");
    if (theta > 0.0 && ctx->prec != FTK_DF) return fail(ctx, FTK_EINVAL, "relaxation needs precision FTK_DF");
    ctx->relax = theta;
    return FTK_OK;
}

ftk_status ftk_autotune(ftk_ctx *ctx, int32_t n_rhs, int32_t which, int32_t *tile_bits_out, int32_t *cols_out,
                        double *us_out) {
    ftk_status s = check_ready(ctx);
    if (s) return s;
    if (n_rhs < 1 || n_rhs > ctx->max_rhs || (n_rhs & (n_rhs - 1)) || (which != 0 && which != 1) ||
        (which == 1 && n_rhs != 1))
        return fail(ctx, FTK_EINVAL, "ftk_autotune: n_rhs must be a power of two <= max_rhs (1 for which = 1)");
    const int prec = which == 1 ? 0 : ctx->mprec;
    const size_t es = elem_bytes(prec);
    // scratch: two Krylov regions (each max_rhs vectors of the vector precision)
    void *in = wsp(ctx, ctx->L.kry[0]);
    void *out = wsp(ctx, ctx->L.kry[1]);
    CK(cudaMemsetAsync(in, 0, ctx->dim * es * n_rhs, ctx->stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double best_us = 1e300;
    Plan best;
    EpiArgs ea{};
    if (prec == 2) ea.df_lo = (long long)n_rhs * (long long)ctx->dim;
    ftk_status st = FTK_OK;
    for (int bc = 1; bc <= std::min((int)n_rhs, hv_max_b(prec)) && st == FTK_OK; bc <<= 1) {
        const int tb_max = std::min(hv_max_tile_bits(prec, bc), ctx->n);
        for (int tb = std::max(5, tb_max - 2); tb <= tb_max && st == FTK_OK; ++tb) {
            Plan pl;
            if (!plan_passes(ctx, prec, bc, tb, pl)) continue;
            for (int rep = 0; rep < 4; ++rep) {
                if (rep == 1 && cudaEventRecord(e0, ctx->stream) != cudaSuccess) st = FTK_ECUDA;
                for (size_t p = 0; p < pl.passes.size() && st == FTK_OK; ++p)
                    if (launch_hv_pass(prec, n_rhs, EPI_PLAIN, in, out, pl.passes[p], ea, pl.grid, ctx->stream) !=
                        cudaSuccess)
                        st = FTK_ECUDA;
            }
            float ms = 0;
            if (st == FTK_OK && (cudaEventRecord(e1, ctx->stream) != cudaSuccess ||
                                 cudaEventSynchronize(e1) != cudaSuccess ||
                                 cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                st = FTK_ECUDA;
            const double us = 1e3 * ms / 3;
            if (st == FTK_OK && us < best_us) { best_us = us; best = pl; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != FTK_OK) return fail(ctx, st, "ftk_autotune: CUDA error while timing");
    if (best.passes.empty()) return fail(ctx, FTK_EINVAL, "ftk_autotune: no admissible plan");
    ctx->plans[prec * 64 + n_rhs] = best;
    if (tile_bits_out) *tile_bits_out = best.tile_bits;
    if (cols_out) *cols_out = best.passes[0].cols;
    if (us_out) *us_out = best_us;
    return FTK_OK;
}

ftk_status ftk_suggest_order(int32_t n_sites, const ftk_bond *bonds, int32_t n_bonds, int32_t precision,
                             int32_t n_rhs, int32_t tile_bits, int32_t *perm_out, int32_t *n_passes_out) {
    if (n_sites < 2 || n_sites > FTK_MAX_SITES || !bonds || n_bonds < 1 || n_bonds > 2 * FTK_MAX_PASS_BONDS ||
        precision < FTK_FP64 || precision > FTK_DF || n_rhs < 1 || n_rhs > FTK_MAX_RHS ||
        (n_rhs & (n_rhs - 1)) || !perm_out)
        return fail(nullptr, FTK_EINVAL, "ftk_suggest_order: bad arguments");
    PlanBond pb[2 * FTK_MAX_PASS_BONDS];
    for (int q = 0; q < n_bonds; ++q) {
        const ftk_bond &b = bonds[q];
        if (b.i < 0 || b.j < 0 || b.i >= n_sites || b.j >= n_sites || b.i == b.j || b.gamma < 0 || b.gamma > 2)
            return fail(nullptr, FTK_EINVAL, "ftk_suggest_order: bond out of range");
        pb[q] = {b.i, b.j, b.gamma};
    }
    const int prec = precision == FTK_FP64 ? 0 : precision == FTK_DF ? 2 : 1;
    const int tb_max = hv_max_tile_bits(prec, n_rhs);
    int tb = tile_bits > 0 ? std::min((int)tile_bits, tb_max) : tb_max;
    tb = std::max(2, std::min(tb, (int)n_sites));
    int perm[FTK_MAX_SITES];
    const int np = plan_suggest_order(n_sites, pb, n_bonds, elem_bytes(prec), std::min((int)n_rhs, hv_max_b(prec)), tb,
                                      perm);
    if (np == 0) return fail(nullptr, FTK_EINVAL, "ftk_suggest_order: planning failed");
    for (int s = 0; s < n_sites; ++s) perm_out[s] = perm[s];
    if (n_passes_out) *n_passes_out = np;
    return FTK_OK;
}

int64_t ftk_launch_count(const ftk_ctx *ctx) { return ctx ? ctx->launches : -1; }

const char *ftk_last_error(const ftk_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_err.c_str(); }

void ftk_destroy(ftk_ctx *ctx) {
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    std::lock_guard<std::mutex> lk(device_mu());
    if (ctx->dsmall) cudaFree(ctx->dsmall);
    if (ctx->stats) cudaFree(ctx->stats);
    if (ctx->shell_scale) cudaFree(ctx->shell_scale);
    if (ctx->slot_energy) cudaFree(ctx->slot_energy);
    if (ctx->slot_norm2) cudaFree(ctx->slot_norm2);
    if (ctx->cocg_exec) cudaGraphExecDestroy(ctx->cocg_exec);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

}  // extern "C"
