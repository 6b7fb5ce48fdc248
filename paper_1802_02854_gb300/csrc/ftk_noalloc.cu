// One mTPQ step through an entry point that allocates nothing.
//
// Who needs it: callers that must not allocate device memory. Examples are
// latency-bound loops that cannot afford the device-wide synchronisation a
// cudaMalloc or cudaFree may imply, and processes whose device memory has
// been handed entirely to a pool that another framework owns, where a
// cudaMalloc would fail. Such a caller cannot create an ftk_ctx (ftk_create
// allocates a few small device buffers), so this entry point takes the
// Hamiltonian and two caller-owned device vectors directly.
//
// Scratch: the per-CTA reduction partials, the last-CTA ticket, the reduced
// dots and the step's scalars live in the file-scope array below (statically
// sized; every GPU that loads the library holds it until the process exits).
// Host code cannot use the array's name as a device address, so the first
// call on each device looks the address up with cudaGetSymbolAddress (that
// device current) and caches it. Every call shares the array and finds the
// previous call's contents in it; the parts that must start at zero are
// cleared on the stream first. Calls whose work overlaps on the GPU race on
// the array.
#include "../../include/ftk.h"
#include "ftk_common.cuh"
#include "ftk_kernels.h"
#include "ftk_plan.h"

#include <algorithm>
#include <cmath>

using namespace ftk;

namespace {

// Largest persistent grid of the H.v passes this entry point launches.
constexpr int kNoallocMaxGrid = FTK_NOALLOC_MAX_GRID;

struct NoallocScratch {
    TpqState tpq;
    unsigned int counter;
    unsigned int pad[3];
    double result[4];
    double stats[3];                       // u_k, logQ_k, <H^2>_k of the step
    double partials[kNoallocMaxGrid * 2];  // [grid][2] per-CTA dots
};

}  // namespace

// The scratch itself (about 16 KB).
static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

namespace {

constexpr int kMaxDevices = 64;
NoallocScratch *g_scratch_ptr[kMaxDevices];   // device address per device, set once
ftk_status noalloc_fail(ftk_status s, const char *m) {
    set_thread_error(m);   // readable through ftk_last_error(NULL)
    return s;
}

}  // namespace

extern "C" ftk_status ftk_tpq_step_noalloc(int32_t n_sites, const ftk_bond *bonds, int32_t n_bonds,
                                           double K, double J, double ell, const void *psi_dev,
                                           void *out_dev, double *stats_out, void *cuda_stream) {
    if (n_sites < 2 || n_sites > FTK_NOALLOC_MAX_SITES)
        return noalloc_fail(FTK_EINVAL, "ftk_tpq_step_noalloc: n_sites must be in [2, FTK_NOALLOC_MAX_SITES]");
    if (!bonds || n_bonds < 1 || n_bonds > 2 * FTK_MAX_PASS_BONDS || !psi_dev || !out_dev || !stats_out ||
        psi_dev == out_dev || !std::isfinite(K) || !std::isfinite(J) || !std::isfinite(ell))
        return noalloc_fail(FTK_EINVAL, "ftk_tpq_step_noalloc: bad arguments");
    // the same rule as ftk_tpq_init: l >= l_min = (1/N) sum_b lambda_max(h_b),
    // with the bond spectrum (J+K)/4 (twice), (J-K)/4, -(3J+K)/4, so that
    // l - H/N is positive semidefinite (Appendix A)
    const double lmax = std::max(std::max((J + K) / 4, (J - K) / 4), -(3 * J + K) / 4);
    const double ell_min = n_bonds * lmax / n_sites;
    if (!(ell >= ell_min - 1e-12))
        return noalloc_fail(FTK_EINVAL, "ftk_tpq_step_noalloc: ell below l_min = (1/N) sum_b lambda_max(h_b)");
    if (((uintptr_t)psi_dev | (uintptr_t)out_dev) & 15)
        return noalloc_fail(FTK_EINVAL, "ftk_tpq_step_noalloc: vectors must be 16-byte aligned");
    PlanBond pb[2 * FTK_MAX_PASS_BONDS];
    for (int q = 0; q < n_bonds; ++q) {
        const ftk_bond &b = bonds[q];
        if (b.i < 0 || b.j < 0 || b.i >= n_sites || b.j >= n_sites || b.i == b.j || b.gamma < 0 || b.gamma > 2)
            return noalloc_fail(FTK_EINVAL, "ftk_tpq_step_noalloc: bond out of range");
        pb[q] = {b.i, b.j, b.gamma};
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return noalloc_fail(FTK_ECUDA, "cudaGetDevice failed");
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return noalloc_fail(FTK_ECUDA, cudaGetErrorString(e));
        e = init_kernel_attributes();
        if (e != cudaSuccess) return noalloc_fail(FTK_ECUDA, cudaGetErrorString(e));
        g_scratch_ptr[dev] = (NoallocScratch *)p;
    }
    NoallocScratch *s = g_scratch_ptr[dev];
    cudaStream_t st = (cudaStream_t)cuda_stream;

    // plan (stack only): FP64, one vector
    PassDesc pd[FTK_MAX_PASSES];
    int tb = 0, cb = 0;
    const int np = plan_hv_passes(n_sites, pb, n_bonds, K, J, 16, 1, hv_max_tile_bits(0, 1), pd, FTK_MAX_PASSES,
                                  &tb, &cb);
    if (np == 0) return noalloc_fail(FTK_EINVAL, "ftk_tpq_step_noalloc: pass planning failed");
    for (int p = 0; p < np; ++p)
        if (!hv_layout_pass(pd[p], 0, 1)) return noalloc_fail(FTK_EINVAL, "ftk_tpq_step_noalloc: pass layout failed");
    const long grid = kNoallocMaxGrid;   // the launcher trims it to the resident CTAs

    // state of this step: normalised input (scale 1), log Q and k start at 0;
    // the ticket must start at zero
    TpqState h{};
    h.scale = 1.0;
    h.ell = ell;
    h.n_sites = n_sites;
    e = cudaMemcpyAsync(&s->tpq, &h, sizeof h, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(&s->counter, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return noalloc_fail(FTK_ECUDA, cudaGetErrorString(e));

    EpiArgs ea{};
    ea.scale = &s->tpq.scale;
    ea.ell = ell;
    ea.inv_n = 1.0 / n_sites;
    ea.partials = s->partials;
    ea.counter = &s->counter;
    ea.result = s->result;
    ea.tpq = &s->tpq;
    ea.stat_u = &s->stats[0];
    ea.stat_logq = &s->stats[1];
    ea.stat_h2 = &s->stats[2];
    for (int p = 0; p < np; ++p) {
        e = launch_hv_pass(0, 1, p == np - 1 ? EPI_TPQ : EPI_PLAIN, psi_dev, out_dev, pd[p], ea, (int)grid, st);
        if (e != cudaSuccess) return noalloc_fail(FTK_ECUDA, cudaGetErrorString(e));
    }
    // q_k = 1 / (new scale); copy u_k, <H^2>_k and q_k back
    double host[3];
    double sc = 0;
    e = cudaMemcpyAsync(host, s->stats, sizeof host, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&sc, &s->tpq.scale, sizeof sc, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return noalloc_fail(FTK_ECUDA, cudaGetErrorString(e));
    stats_out[0] = host[0];
    stats_out[1] = host[2];
    stats_out[2] = 1.0 / sc;
    return FTK_OK;
}
