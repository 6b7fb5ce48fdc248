/*
 * ftk.h -- C-ABI of the GB300 FTKomega hot path.
 *
 * Method: Yamaji, Suzuki, Kawamura, "Finite-temperature spectra of quantum
 * lattice models by the shifted Krylov method and typical pure states"
 * (arXiv:1802.02854). Every entry point cites the passage that defines the
 * operation it performs.
 *
 * Conventions shared by all entry points
 * -------------------------------------
 * Basis (Sec. II.A): |x> = |sigma_0 ... sigma_{N-1}>, bit l of the index x is
 *   site l, bit 1 = spin up. A state is 2^N complex amplitudes in index order.
 * Precision: FTK_FP64 stores complex amplitudes as two doubles (16 B),
 *   FTK_FP32 as two floats (8 B). FTK_MIXED keeps FP64 shells, probes and
 *   Krylov residuals (the residuals as float hi + lo pairs, 16 B) and runs
 *   H.v in FP32 on the hi parts, with the COCG dot mu = r^T H r taken from
 *   hi + lo; its accuracy follows the FP32 matvec (relative 1e-7 per
 *   product), not the FP32 rounding of the recurrence. All scalar inputs and
 *   outputs are double in every mode; TPQ statistics, Krylov scalars and
 *   reweighting sums are computed in double; the per-thread partial sums of
 *   norms and inner products are double (FTK_FP64), compensated float
 *   (FTK_FP32) or double-float pairs (the COCG dots of FTK_MIXED / FTK_DF),
 *   and are reduced across threads in double.
 *   FTK_DF is the mixed mode with H.v in double-float arithmetic on the FP32
 *   pipe (hi + lo float pairs in and out, ~48 bits): FP64-class accuracy at
 *   the FP32 pipe's issue rate; its residual update runs inside the first H.v
 *   pass of the next step. The mTPQ state is FP64 in every mode.
 * Memory: device vectors live in ONE caller-allocated device workspace
 *   (ftk_footprint gives its size, ftk_bind_workspace hands it over); the
 *   library never allocates vector-sized memory itself. The context owns only
 *   a few small device buffers (constants, scalars, reduction flags).
 *   Host arrays are owned by the caller and only read/written during a call.
 * Streams: all device work of a context is issued on opts.cuda_stream
 *   (NULL = legacy default stream). Calls that return host results
 *   synchronise that stream; the others are asynchronous.
 * Threading: a context is used from one host thread at a time.
 * Errors: every call returns an ftk_status; FTK_OK == 0. No exception or
 *   longjmp crosses the ABI. ftk_last_error() returns a message for the last
 *   failing call on that context. After FTK_ECUDA the context should be
 *   destroyed.
 */
#ifndef FTK_H
#define FTK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ftk_ctx ftk_ctx;

typedef enum {
    FTK_OK = 0,
    FTK_EINVAL = 1,       /* invalid argument (message says which)              */
    FTK_ENOMEM = 2,       /* workspace missing or too small                      */
    FTK_ECUDA = 3,        /* a CUDA call failed                                  */
    FTK_ENOCONV = 4,      /* Krylov solve hit max_iter; outputs still written    */
    FTK_EBREAKDOWN = 5,   /* COCG breakdown (r^T r or p^T A p vanished)          */
    FTK_ETIMEOUT = 6,     /* a bounded device wait gave up                       */
    FTK_ETRUNC = 7,       /* reweighting series truncated for some temperature   */
    FTK_EBUSY = 8         /* context busy / state missing for the request        */
} ftk_status;

enum { FTK_FP64 = 0, FTK_FP32 = 1, FTK_MIXED = 2, FTK_DF = 3 };
enum { FTK_GAMMA_X = 0, FTK_GAMMA_Y = 1, FTK_GAMMA_Z = 2 };

/* Cluster geometry: n_sites sites, pos[2*l], pos[2*l+1] = real-space (x, y)
 * position R_l of site l (Sec. V: R_l is the site position, not the cell's). */
typedef struct {
    int32_t n_sites;
    const double *pos;
} ftk_lattice;

/* One nearest-neighbour bond (i, j) of type gamma in {0=x, 1=y, 2=z}. */
typedef struct {
    int32_t i, j, gamma;
} ftk_bond;

typedef struct {
    int32_t precision;    /* FTK_FP64, FTK_FP32, FTK_MIXED or FTK_DF             */
    int32_t max_rhs;      /* right-hand sides per blocked solve (1..32)          */
    int32_t n_saved;      /* shell states the workspace keeps (>= 1)             */
    int32_t tile_bits;    /* amplitudes per CTA tile = 2^tile_bits; 0 = tuned    */
    void *cuda_stream;    /* cudaStream_t, or NULL for the default stream        */
} ftk_opts;

/* Bytes of device workspace a context with these sizes needs (0 on bad
 * arguments). Layout: 2 TPQ vectors + n_saved shells + max_rhs probe vectors
 * + 3 * max_rhs Krylov vectors + reduction scratch. */
size_t ftk_footprint(int32_t n_sites, int32_t n_saved, int32_t max_rhs, int32_t precision);

/* Build a context for the Kitaev-Heisenberg Hamiltonian (Sec. V.A)
 *   H = sum_<ij>_gamma J S_i.S_j + K S^gamma_i S^gamma_j
 * on the given lattice/bond list. Requires 2 <= n_sites <= 30, bonds with
 * 0 <= i, j < n_sites, i != j, gamma in {0, 1, 2}. Copies everything it needs
 * (the caller may free lattice/bonds afterwards). Plans the tiled H.v passes
 * (bonds whose two sites share a tile are applied in shared memory).
 * On success *out receives the context. */
ftk_status ftk_create(const ftk_lattice *lattice, const ftk_bond *bonds, int32_t n_bonds,
                      double K, double J, const ftk_opts *opts, ftk_ctx **out);

/* Hand the context a device workspace of at least ftk_footprint(...) bytes,
 * 256-byte aligned. The caller keeps ownership and must keep it alive until
 * ftk_destroy or the next bind. Rebinding discards TPQ and Krylov state. */
ftk_status ftk_bind_workspace(ftk_ctx *ctx, void *dev_ptr, size_t bytes);

/* Seeded random initial state (Sec. II.A): c_x complex Gaussian, normalised
 * (uniform on the unit sphere of R^{2 N_F}). Counter-based Philox4x32-10
 * (Salmon et al. 2011): element x uses counter (x_lo, x_hi, sample, 0) and key
 * (seed_lo, seed_hi); u1, u2 from the two 64-bit halves (>> 11, + 0.5, * 2^-53);
 * Box-Muller c_x = sqrt(-2 ln u1) exp(2 pi i u2). Generated in double, stored
 * in the context precision. ell is the mTPQ constant l of Eq. B1; it must be
 * >= l_min = (1/N) sum_b lambda_max(h_b) so that l - H/N is positive
 * semidefinite (else FTK_EINVAL). Resets the step counter to k = 0. */
ftk_status ftk_tpq_init(ftk_ctx *ctx, uint64_t seed, uint32_t sample, double ell);

/* Set the TPQ state to a caller vector (normalised by the call), e.g. for
 * parity runs. v: 2^N complex amplitudes as interleaved (re, im) doubles,
 * host (is_device = 0) or device (is_device = 1) memory. Same ell rules and
 * reset as ftk_tpq_init. */
ftk_status ftk_set_state(ftk_ctx *ctx, const double *v, int32_t is_device, double ell);

/* n_steps mTPQ iterations (Appendix A, the (l - h)^k building block of
 * Eq. B1): psi_{k+1} = (l - H/N) psi_k / q_k. For each input state k (from
 * the current step on) the host arrays (length n_steps, may be NULL) receive
 *   u_out[i]    = <psi_k|H|psi_k> / N
 *   logQ_out[i] = log ||(l - H/N)^k psi_0||
 *   h2_out[i]   = <psi_k|H^2|psi_k>
 * and psi_k is kept as shell number k / save_every when k % save_every == 0
 * (at most n_saved shells; FTK_ENOMEM if more are needed). Synchronises. */
ftk_status ftk_tpq_step(ftk_ctx *ctx, int32_t n_steps, int32_t save_every,
                        double *u_out, double *logQ_out, double *h2_out);

/* Number of shells saved so far and, per shell, its step k and energy
 * E_k = N u_k (host arrays of length >= n_saved, may be NULL). */
ftk_status ftk_shells(const ftk_ctx *ctx, int32_t *n_out, int32_t *step_out, double *energy_out);

/* Probe vector for the dynamical structure factor (Sec. V, S^alpha_{+Q}):
 *   lambda = N^{-1/2} sum_l exp(+i q.R_l) S^gamma_l psi_shell
 * written to probe slot rhs_slot (0 <= rhs_slot < max_rhs). q[2] is the
 * momentum in the lattice's Cartesian frame. The slot remembers its shell
 * (its energy sets the shift origin of ftk_shifted_cocg). Asynchronous. */
ftk_status ftk_apply_op(ftk_ctx *ctx, int32_t shell, int32_t gamma, const double q[2],
                        int32_t rhs_slot);

/* Load probe slot rhs_slot with a caller vector lambda (host or device, same
 * layout as ftk_set_state, not normalised) whose shift origin is energy. */
ftk_status ftk_set_probe(ftk_ctx *ctx, int32_t rhs_slot, const double *v, int32_t is_device,
                         double energy);

/* Shifted COCG (Sec. II.B; BiCG with shadow conj(r) on the complex-symmetric
 * z - H, Frommer 2003 for the shifts) for the probes in rhs_slots[0..n_rhs):
 *   G_j(omega_s) = <lambda_j| (z_js - H)^{-1} |lambda_j>,  z_js = E_j + omega_s + i eta
 * with E_j the slot's shift origin. The n_rhs solves run as one blocked
 * iteration (one H.V over all of them per step) with per-RHS scalars; the
 * seed shift of RHS j is z_j at omega[n_omega/2]. Solve j stops at the first
 * iteration with max_s ||r_j|| / |pi_js| <= tol ||lambda_j||.
 * G_out: host, [n_rhs][n_omega] complex as (re, im) doubles. iters_out: host
 * [n_rhs] (may be NULL). Returns FTK_ENOCONV if some solve hit max_iter
 * (G still written), FTK_EBREAKDOWN on breakdown. n_omega <= 4096. Synchronises. */
ftk_status ftk_shifted_cocg(ftk_ctx *ctx, const int32_t *rhs_slots, int32_t n_rhs,
                            const double *omega, int32_t n_omega, double eta,
                            double tol, int32_t max_iter,
                            double *G_out, int32_t *iters_out);

/* Options of ftk_shifted_cocg_ex (a NULL pointer selects the defaults). */
typedef struct {
    /* Probe slots of the projection vectors, one per right-hand side: the
     * solve then returns G^{AB}(z) = <lambda_A|(z - H)^{-1}|lambda_B> with
     * lambda_B in rhs_slots[j] and lambda_A in proj_slots[j] (the A != B
     * response of Sec. II.B, e.g. cross correlations of two operators).
     * NULL: A = B. */
    const int32_t *proj_slots;
    /* Shift whose system is the initial seed; -1: n_shift / 2. */
    int32_t seed_index;
    /* 1: seed switching. When the seed system has converged while other
     * shifts have not, the unconverged shift with the largest residual
     * ||r_k|| / |pi^s_k| becomes the seed (the seed is moved as the
     * truncation criterion of Appendix C follows the largest residual).
     * Only residuals enter the recurrences, so the switch is an exact
     * rescaling (r_k / pi*_k, r_{k-1} / pi*_{k-1}, pi / pi*): G and every
     * shifted residual are unchanged, and a seed that converges early no
     * longer drives its residual toward underflow. */
    int32_t seed_switch;
} ftk_cocg_opts;

/* Shifted COCG as ftk_shifted_cocg with general complex shifts and the
 * options above: G_j(s) = <lambda_{A,j}|(E_j + z_s - H)^{-1}|lambda_{B,j}>
 * for shifts[2 s] + i shifts[2 s + 1] (host, [n_shift][2], imaginary parts
 * > 0), E_j the shift origin of rhs slot j. switches_out (host [n_rhs], may
 * be NULL) receives the number of seed switches per right-hand side. Other
 * arguments, outputs, errors and synchronisation as ftk_shifted_cocg. */
ftk_status ftk_shifted_cocg_ex(ftk_ctx *ctx, const int32_t *rhs_slots, int32_t n_rhs, const double *shifts,
                               int32_t n_shift, double tol, int32_t max_iter, const ftk_cocg_opts *opts,
                               double *G_out, int32_t *iters_out, int32_t *switches_out);

/* Canonical TPQ states (Appendix A, Eq. B1) at the inverse temperatures
 * beta[0..n_beta) (finite, >= 0, ascending):
 *   |phi_b> = exp(N b (l - h)/2) |psi> / ||.||,   h = H / N,
 * psi the current TPQ state (normalised), l the context's ell. Each
 * increment db = beta[i] - beta[i-1] (beta[-1] = 0) is applied in M_d steps
 * of the Taylor series of exp(tau (l - h)), tau = N db / (2 M_d), with M_d
 * from the fixed point X of X_{j+1} = ln lam + ln(2 pi X_j) / 2 (X_0 = lam,
 * so that the largest term of a step is about lam):
 *   M_d = ceil(N db (l + |eps_0|) / (2 X)),  |eps_0| <= (1/N) sum_b |lambda_min(h_b)|;
 * a step stops at the first term k >= X with X^k / k! <= 1e-17 (then the
 * rest is below 1e-17 of the sum, l - h being positive semidefinite).
 * Outputs (host, [n_beta], may be NULL): log ||exp(N b (l - h)/2) psi||,
 * M_d of the increment, and the energy <phi_b|H|phi_b>. phi_b is kept as
 * shell first_shell + i (scale 1; its shift origin is that energy), and the
 * TPQ state becomes the last phi_b with the step counter reset to 0.
 * Needs the Krylov region to hold two FP64 vectors (FTK_ENOMEM else) and
 * first_shell + n_beta <= n_saved; lam > 1. Synchronises. */
ftk_status ftk_ctpq(ftk_ctx *ctx, const double *beta, int32_t n_beta, double lam, int32_t first_shell,
                    double *log_norm_out, int32_t *md_out, double *energy_out);

/* Bytes of device scratch ftk_filter_shells needs for n_centres shells of
 * n_points contour points each and at most max_iter Krylov iterations:
 * 48 B per (iteration, contour point) of recorded shift recurrences plus
 * 16 B per (iteration, shell) of coefficients. 0 on bad arguments
 * (n_points <= 32, n_centres * n_points <= 4096). */
size_t ftk_filter_footprint(int32_t n_centres, int32_t n_points, int32_t max_iter);

/* Filtered typical states (Sec. II.C, Eq. dfilterP and Eq. filtered):
 *   phi^m = P_{E_m, eps, M} phi
 *         = (1/M) sum_{j=1..M} eps e^{i th_j} (eps e^{i th_j} + E_m - H)^{-1} phi,
 *   th_j = 2 pi (j - 1/2) / M,  E_m = e_b + (2m + 1) eps,  m < n_centres,
 * phi the normalised source: src = 0 the current TPQ state, src = 1 + s
 * shell s (e.g. a cTPQ state from ftk_ctpq). All n_centres * M resolvents
 * share phi, so one shifted COCG over all contour points runs twice: the
 * first pass records the shift recurrences in scratch (caller-owned device
 * memory of ftk_filter_footprint bytes, 256-byte aligned), the second
 * replays the solve and accumulates each phi^m from the residuals with the
 * coefficients of x^s = sum_k (T^s_k / pi^s_k) r_k. phi^m is written to
 * shell first_shell + m (not normalised; its shift origin is E_m), probe
 * slot 0 is overwritten (it holds phi). norm2_out (host [n_centres], may
 * be NULL) receives <phi^m|phi^m>, iters_out (may be NULL) the iterations
 * of one pass. The solve stops when every contour residual is below
 * tol ||phi||. Needs precision FTK_FP64 and first_shell + n_centres <=
 * n_saved. FTK_ENOCONV if max_iter is reached (no shells written).
 * Synchronises. */
ftk_status ftk_filter_shells(ftk_ctx *ctx, int32_t src, double e_b, double eps, int32_t n_centres,
                             int32_t n_points, double tol, int32_t max_iter, void *scratch_dev,
                             size_t scratch_bytes, int32_t first_shell, double *norm2_out,
                             int32_t *iters_out);

/* Reweighting of filter shells (Sec. II.D, Eqs. FRW1 and FRW2): with
 * b' = 1 / T[t] and n_m = norm2[m] = <phi^m|phi^m> of shells built at
 * inverse temperature beta,
 *   S(omega, T) = sum_m e^{(b - b') E_m} S_m(omega) / sum_l e^{(b - b') E_l} n_l,
 *   S_m(omega)  = -Im G_m(omega) / pi,
 *   P_T(E_m)    = e^{(b - b') E_m} n_m / (2 eps sum_l e^{(b - b') E_l} n_l),
 * G: host [n_shell][n_omega] complex (re, im), the Green's functions of the
 * filtered shells (Eq. GAB_TPS: <phi^m|A^dag (omega + i eta + E_m - H)^{-1} A|phi^m>,
 * e.g. ftk_apply_op on the shell then ftk_shifted_cocg); energy: host
 * [n_shell] E_m. S_out: host [n_T][n_omega]; P_out: host [n_T][n_shell]
 * (may be NULL). Computed on the device in double with log-sum-exp.
 * Synchronises. */
ftk_status ftk_filter_spectrum(ftk_ctx *ctx, const double *G, int32_t n_shell, int32_t n_omega,
                               const double *energy, const double *norm2, double beta, double eps,
                               const double *T, int32_t n_T, double *S_out, double *P_out);

/* Temperature sweep by reweighting the saved shells (reading R1 of the
 * Taylor series Eq. B1; the shell-to-temperature map of Sec. III.D):
 *   S(omega, T) = sum_s W_s(1/T) S_s(omega) / sum_s W_s(1/T),
 *   S_s(omega) = -Im G_s(omega) / pi,
 * with W_s the sum of the series weights w_n whose step floor(n/2) is nearest
 * to shell s (ties to the later shell). G: host [n_shell][n_omega] complex
 * (re, im) for shells 0..n_shell-1 of this context (their TPQ statistics are
 * kept by the context). S_out: host [n_T][n_omega]. trunc_out: host [n_T]
 * (may be NULL), 1 where the series tail exceeds 1e-14 of the total; then the
 * call returns FTK_ETRUNC with S still written. Computed on the device in
 * double. Synchronises. */
ftk_status ftk_spectrum(ftk_ctx *ctx, const double *G, int32_t n_shell, int32_t n_omega,
                        const double *T, int32_t n_T, double *S_out, int32_t *trunc_out);

/* ftk_spectrum with the mTPQ statistics given by the caller instead of the
 * context's sequence (the same reading R1 of Eq. B1): u[k] = u_k, logQ[k] =
 * log Q_k for k < n_steps (host), shells s at steps s save_every, l = ell.
 * For statistics merged from momentum sectors (ftk_sector_combine) or kept
 * from an earlier TPQ sequence. Requires l > u_k and (n_shell - 1) save_every
 * < n_steps <= 262144. Other arguments and outputs as ftk_spectrum. */
ftk_status ftk_spectrum_ex(ftk_ctx *ctx, const double *G, int32_t n_shell, int32_t n_omega, const double *T,
                           int32_t n_T, const double *u, const double *logQ, int32_t n_steps, int32_t save_every,
                           double ell, double *S_out, int32_t *trunc_out);

/* ---------------------------------------------------------------------------
 * Momentum sectors (translation symmetry). The paper works in the full basis
 * (Sec. V); a sector reduces the dimension by the number of translations
 * (N/2) for larger clusters. A group of site permutations g (element 0 the
 * identity; each must map the bond list of the context to itself) acts on
 * basis states, bit g(l) of g.x = bit l of x, and commutes with H. A sector
 * is a unitary one-dimensional character chi of the group (for the torus
 * translation by a_g at momentum Q: chi(g) = exp(-i Q.a_g)); its basis
 * vectors are |r>_chi = sqrt(o_r) P|r>, P = (1/|G|) sum_g chi(g)^* g, for the
 * orbit representatives r (smallest integer of the orbit, o_r its size) on
 * whose stabiliser chi is 1. A sector vector holds dim complex amplitudes
 * (FP64 (re, im)) in ascending order of r.
 * The sector owns its device memory (allocated by ftk_sector_create): 4 B per
 * full-basis state for the state -> (orbit, element) table, the orbit list,
 * and n_slots sector vectors; 9 B per full-basis state of temporary memory
 * during creation. Work runs on the context's stream.
 * ------------------------------------------------------------------------- */
typedef struct ftk_sector ftk_sector;

/* perms: host [n_g][n_sites] (site l -> perms[g][l]), 1 <= n_g <= 32; chi: host
 * [n_g][2] (re, im). n_slots: sector vectors kept (1..64). *dim_out
 * receives the sector dimension. FTK_EINVAL if the permutations do not form
 * a group preserving the bonds, or chi is not a character of it. */
ftk_status ftk_sector_create(ftk_ctx *ctx, const int32_t *perms, int32_t n_g, const double *chi, int32_t n_slots,
                             ftk_sector **out, int64_t *dim_out);
void ftk_sector_destroy(ftk_sector *sector);

/* Dimension, number of orbits of the group, and (host [dim], may be NULL) the
 * representative of every sector basis vector. Synchronises. */
ftk_status ftk_sector_info(const ftk_sector *sector, int64_t *dim, int32_t *n_orbits, uint32_t *reps_host);

/* Copy a sector vector in (host or device) / out (host). Synchronise. */
ftk_status ftk_sector_set(ftk_sector *sector, int32_t slot, const double *v, int32_t is_device);
ftk_status ftk_sector_get(ftk_sector *sector, int32_t slot, double *host_out);

/* Components of a full-basis state in the sector: slot[r] = <r|_chi psi =
 * (sqrt(o_r)/|G|) sum_h chi(h)^* psi[h^{-1}.r]. psi: 2^N complex (re, im)
 * doubles, host (is_device = 0) or device. Synchronises. */
ftk_status ftk_sector_project(ftk_sector *sector, const double *psi_full, int32_t is_device, int32_t slot);

/* slot_out = H_chi slot_in (the sector block of the Kitaev-Heisenberg H of the
 * context, Sec. V.A; a gather over the bonds of each representative with the
 * character phases). Asynchronous. */
ftk_status ftk_sector_hv(ftk_sector *sector, int32_t slot_in, int32_t slot_out);

/* mTPQ iteration in the sector (Appendix A): the state in slot_state is
 * normalised (log of its norm to *lognorm0_out, may be NULL), then n_steps
 * times psi_{k+1} = (l - H/N) psi_k / q_k with slot_work as scratch; psi_k is
 * copied to slot first_save_slot + k / save_every when k % save_every == 0.
 * Host outputs (length n_steps, may be NULL): u_out[k] = <psi_k|H|psi_k>/N,
 * logq_out[k] = log of the product of q below k. Sector parts of one full
 * state are merged by ftk_sector_combine. ell >= l_min as ftk_tpq_init.
 * Synchronises. */
ftk_status ftk_sector_tpq(ftk_sector *sector, int32_t slot_state, int32_t slot_work, double ell, int32_t n_steps,
                          int32_t save_every, int32_t first_save_slot, double *u_out, double *logq_out,
                          double *lognorm0_out);

/* lambda = S^z_q psi (Sec. V) from sector src to sector dst, which must be
 * src's sector shifted by q (chi_dst(g) = chi_src(g) exp(-i q.a_g), checked
 * on the translation of site 0): S^z_q keeps the representative,
 * lambda[r] = f_q(r) psi[r], f_q(r) = N^{-1/2} sum_l e^{i q.R_l} s_l(r)/2.
 * Synchronises. */
ftk_status ftk_sector_apply_sz(ftk_sector *src, int32_t slot_src, ftk_sector *dst, int32_t slot_dst,
                               const double q[2]);

/* G(z_s) = <lambda|(z_s - H_chi)^{-1}|lambda> for lambda in slot and the
 * complex shifts z_s (host [n_shift][2]): the Hermitian Lanczos process on
 * H_chi (a sector block is complex Hermitian, so the bilinear COCG does not
 * apply) with the shifted recurrences of the LDL^T factors of z - T_j,
 *   d_j = z - a_j - b_j^2/d_{j-1},  y_j = y_{j-1} b_j/d_{j-1},
 *   G_j = |lambda|^2 sum_i y_i^2/d_i;
 * a shift stops once |b_{j+1} y_j/d_j| <= tol (its residual relative to
 * |lambda|, the criterion of ftk_shifted_cocg). The three slots after `slot`
 * (cyclically; n_slots >= 4) are overwritten. G_out: host [n_shift][2];
 * iters_out: Lanczos steps. FTK_ENOCONV at max_iter (G written).
 * Synchronises. */
ftk_status ftk_sector_green(ftk_sector *sector, int32_t slot, const double *shifts, int32_t n_shift, double tol,
                            int32_t max_iter, double *G_out, int32_t *iters_out);

/* Merge the sector parts of one full-space mTPQ sequence (host arithmetic):
 * with a_s[k] = lognorm0[s] + logq[s][k], the full statistics
 *   logQ_out[k] = (1/2) log sum_s e^{2 a_s[k]} - (1/2) log sum_s e^{2 lognorm0[s]},
 *   u_out[k]    = sum_s e^{2 a_s[k]} u[s][k] / sum_s e^{2 a_s[k]},
 * and the Green's functions of the normalised full shells
 *   G_out[i] = sum_s e^{2 a_s[k_i]} G[s][i] / sum_s e^{2 a_s[k_i]},  k_i = shell_steps[i],
 * from each sector's G of its normalised shell (S^z_q maps each sector to
 * one sector, so the sector blocks of the resolvent add). Arrays host:
 * lognorm0 [n_sec], logq and u [n_sec][n_steps], G [n_sec][n_shell][n_omega][2],
 * outputs u_out, logQ_out [n_steps], G_out [n_shell][n_omega][2]. */
ftk_status ftk_sector_combine(int32_t n_sec, int32_t n_steps, const double *lognorm0, const double *logq,
                              const double *u, int32_t n_shell, const int32_t *shell_steps, int32_t n_omega,
                              const double *G, double *u_out, double *logQ_out, double *G_out);

/* out = H v for n_rhs vectors stored one after the other (layout
 * [n_rhs][2^N] complex in the matvec precision: FP64 for FTK_FP64, FP32 for
 * FTK_FP32 and FTK_MIXED; vector j at offset j 2^N; for FTK_DF the FP32 hi
 * parts [n_rhs][2^N] followed by the lo parts [n_rhs][2^N], value hi + lo).
 * v and out are device pointers, must not overlap, and
 * need 16-byte alignment. The product of Sec. IV.A's cost unit ("a Lanczos
 * step"); exposed for tests and the bandwidth metric. Asynchronous. */
ftk_status ftk_hv(ftk_ctx *ctx, const void *v_dev, void *out_dev, int32_t n_rhs);

/* Copy 2^N amplitudes of an internal vector to the host as (re, im) doubles:
 * which = 0 current TPQ state (normalised), 1 + s shell s (normalised),
 * -1 - j probe slot j. Synchronises. */
ftk_status ftk_get_vector(ftk_ctx *ctx, int32_t which, double *host_out);

/* Number of H.v passes the plan uses, and the tile bits. */
ftk_status ftk_plan_info(const ftk_ctx *ctx, int32_t *n_passes, int32_t *tile_bits);

/* Site relabelling that lets H.v run in fewer tiled passes (the layout
 * choice of Sec. IV.A's Hamiltonian-vector product on this hardware: the
 * chunk sites, i.e. the lowest index bits, sit in every tile). Host only, no
 * device work. bonds as in ftk_create; precision and n_rhs select the tile
 * shape (tile_bits 0 = the default). perm_out (host, n_sites ints) receives
 * site l -> new label perm_out[l]; relabel the sites (and their positions)
 * before ftk_create. n_passes_out (may be NULL) receives the pass count.
 * The search is deterministic: seeded choices of the chunk sites with greedy
 * covers, then a bounded local search over the chunk sites and the passes
 * together (about 0.1 s at N = 24). Contexts plan their own passes with the
 * same local search for fixed labels.
 * FTK_EINVAL on bad arguments (message via ftk_last_error(NULL)). */
ftk_status ftk_suggest_order(int32_t n_sites, const ftk_bond *bonds, int32_t n_bonds, int32_t precision,
                             int32_t n_rhs, int32_t tile_bits, int32_t *perm_out, int32_t *n_passes_out);

/* Relaxed double-float solve (context precision FTK_DF only). theta > 0:
 * once every unfinished right-hand side of a ftk_shifted_cocg call has a
 * residual max_s ||r_k|| / |pi^s_k| / ||lambda|| below theta, its remaining
 * matrix-vector products run in FP32 (3-pass FP32 H.V of the hi parts, mu
 * from hi + lo) while the residual recurrence, the dots and the shift
 * recurrences stay double-float / FP64. The product error then enters the
 * shifted residuals scaled by that small residual (inexact Krylov
 * relaxation; the measured spectrum error is stated with the bench). theta =
 * 0 (the default) keeps every product double-float. Returns FTK_EINVAL for a
 * negative or non-finite theta, or theta > 0 on another precision. */
ftk_status ftk_set_relax(ftk_ctx *ctx, double theta);

/* Autotuner of the blocked H.V (the batching knob of the Sec. IV.A product
 * on this hardware). Times, on scratch vectors in the context's Krylov
 * region, every admissible plan for n_rhs right-hand sides: column chunk
 * width (1, 2, 4 or 8 vectors per launch) x tile size (the two to three
 * largest tiles that fit), and installs the fastest one for later ftk_hv,
 * ftk_shifted_cocg (which = 0, the context's matvec precision) or
 * ftk_tpq_step (which = 1, FP64, n_rhs = 1) calls. Outputs (may be NULL):
 * the chosen tile bits and chunk width and its time per H.V in us.
 * n_rhs: a power of two <= max_rhs. Overwrites the Krylov region (call it
 * outside a solve). Synchronises. */
ftk_status ftk_autotune(ftk_ctx *ctx, int32_t n_rhs, int32_t which, int32_t *tile_bits_out, int32_t *cols_out,
                        double *us_out);

/* Kernel launches issued by this context since creation (for accounting). */
int64_t ftk_launch_count(const ftk_ctx *ctx);

/* One mTPQ step that allocates no memory at all (no cudaMalloc/cudaFree, no
 * library allocator). The paper has no counterpart: this is a deployment
 * entry point for callers that cannot allocate device memory, such as
 * latency-bound loops that cannot afford the device-wide synchronisation an
 * allocation may imply, or processes whose device memory is all held by a
 * pool another framework owns (a cudaMalloc would fail there). Such callers
 * cannot use ftk_create, which allocates small device buffers.
 *   out = (l - H/N) psi   (unnormalised; H as in ftk_create)
 * psi_dev, out_dev: caller-owned device vectors of 2^n_sites FP64 complex
 * amplitudes ((re, im) doubles), 16-byte aligned, not overlapping; psi must
 * be normalised. stats_out (host, 3 doubles) receives u = <psi|H|psi>/N,
 * <psi|H^2|psi> and q = ||out||, so out / q is the next mTPQ state.
 * Requires 2 <= n_sites <= FTK_NOALLOC_MAX_SITES and, as ftk_tpq_init,
 * ell >= l_min = (1/N) sum_b lambda_max(h_b); bonds as in ftk_create (else
 * FTK_EINVAL, message via ftk_last_error(NULL)). Work runs on cuda_stream
 * (NULL = the legacy default stream, which waits for every blocking stream);
 * the call copies its three scalars to host memory and synchronises that
 * stream before returning.
 * Scratch: a static device array of about 16 KB per GPU holds the reduction
 * partials of at most FTK_NOALLOC_MAX_GRID CTAs and the step's scalars; the
 * first call on a device looks up its address. All calls share it, so calls
 * whose GPU work overlaps (other threads or streams) race and must be
 * serialised by the caller. */
#define FTK_NOALLOC_MAX_SITES 30
#define FTK_NOALLOC_MAX_GRID 1024
ftk_status ftk_tpq_step_noalloc(int32_t n_sites, const ftk_bond *bonds, int32_t n_bonds,
                                double K, double J, double ell, const void *psi_dev,
                                void *out_dev, double *stats_out, void *cuda_stream);

/* Message of the last failing call on ctx; with ctx == NULL, of the last
 * failing ftk_create on this host thread. Valid until the next call. */
const char *ftk_last_error(const ftk_ctx *ctx);
void ftk_destroy(ftk_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* FTK_H */
