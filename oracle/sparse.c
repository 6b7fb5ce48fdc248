/*
 * Oracle: plain, slow, matrix-free FTKomega in FP64 (C99 + OpenMP).
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library. It shares
 * no code with the CUDA path.
 *
 * Every routine follows a passage of arXiv:1802.02854 (Yamaji, Suzuki,
 * Kawamura) directly; nothing is blocked, fused or reordered beyond what the
 * definition states.
 *
 * Basis (Sec. II.A): |x> = |sigma_0 ... sigma_{N-1}>, bit l of x is site l,
 * bit 1 = up. s_l(x) = +1 for up, -1 for down.
 * Single-spin rules used below (S = sigma/2):
 *   S^z |x> = (s_l/2) |x>
 *   S^x |x> = (1/2)   |x ^ 2^l>
 *   S^y |x> = (i s_l/2) |x ^ 2^l>      (sigma^y|up> = i|down>, sigma^y|down> = -i|up>)
 */
#define _GNU_SOURCE
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define ORC_PI 3.14159265358979323846

static inline int spin(uint64_t x, int l) { return ((x >> l) & 1u) ? 1 : -1; }

/* <y| S^a_i S^a_j |x> for y = x ^ (2^i | 2^j), a in {x, y}: the amplitude of
 * the flipped state produced from |x>. */
static cplx flip_amp(int a, uint64_t x, int i, int j)
{
    if (a == 0) return 0.25;                                   /* S^x S^x */
    return (I * 0.5 * spin(x, i)) * (I * 0.5 * spin(x, j));    /* S^y S^y */
}

/*
 * Kitaev-Heisenberg Hamiltonian (Sec. V.A):
 *   H = sum_<ij>_gamma  J S_i.S_j + K S_i^gamma S_j^gamma
 * applied matrix-free as out_y = sum_x <y|H|x> v_x. Each bond term maps a
 * basis state |x> to a multiple of |x> (S^z S^z) or of |x ^ 2^i ^ 2^j>
 * (S^x S^x, S^y S^y), so only x = y and x = y ^ 2^i ^ 2^j contribute; the
 * matrix element <y|T|x> is obtained by acting with T on the source |x>.
 * Parallel over y. bonds: [n_bonds][3] = (i, j, gamma), gamma 0=x 1=y 2=z.
 */
void orc_hv(int n_sites, int n_bonds, const int32_t *bonds, double K, double J,
            const cplx *v, cplx *out)
{
    int64_t d = (int64_t)1 << n_sites;
    #pragma omp parallel for schedule(static)
    for (int64_t y = 0; y < d; ++y) {
        cplx acc = 0;
        for (int b = 0; b < n_bonds; ++b) {
            int i = bonds[3 * b], j = bonds[3 * b + 1], g = bonds[3 * b + 2];
            uint64_t x = (uint64_t)y ^ (1ull << i) ^ (1ull << j);   /* flipped source */
            /* J S_i.S_j = J (SxSx + SySy + SzSz) */
            acc += J * flip_amp(0, x, i, j) * v[x];
            acc += J * flip_amp(1, x, i, j) * v[x];
            acc += J * 0.25 * spin(y, i) * spin(y, j) * v[y];
            /* K S^gamma S^gamma */
            if (g == 2) acc += K * 0.25 * spin(y, i) * spin(y, j) * v[y];
            else        acc += K * flip_amp(g, x, i, j) * v[x];
        }
        out[y] = acc;
    }
}

static cplx dotc(uint64_t d, const cplx *a, const cplx *b)   /* a^dagger b */
{
    cplx s = 0;
    for (uint64_t x = 0; x < d; ++x) s += conj(a[x]) * b[x];
    return s;
}

static cplx dotu(uint64_t d, const cplx *a, const cplx *b)   /* a^T b (bilinear) */
{
    cplx s = 0;
    for (uint64_t x = 0; x < d; ++x) s += a[x] * b[x];
    return s;
}

/*
 * Microcanonical TPQ iteration (Appendix A, Eq. B1 building block):
 *   psi_{k+1} = (l - H/N) psi_k / q_k,  q_k = ||(l - H/N) psi_k||.
 * For each input state k = 0 .. n_steps-1 it records
 *   u_k     = <psi_k|H|psi_k> / N
 *   logQ_k  = sum_{k'<k} log q_k'       (Q_k = ||(l - h)^k psi_0||)
 *   h2_k    = <psi_k|H^2|psi_k>  = N^2 (q_k^2 - l^2 + 2 l u_k)
 * and stores psi_k as a shell when k % save_every == 0.
 * psi0 must be normalised.
 */
int orc_tpq(int n_sites, int n_bonds, const int32_t *bonds, double K, double J,
            const cplx *psi0, double ell, int n_steps, int save_every,
            cplx *shells, double *u, double *logQ, double *h2)
{
    uint64_t d = 1ull << n_sites;
    double n = (double)n_sites;
    cplx *psi = malloc(d * sizeof(cplx)), *hpsi = malloc(d * sizeof(cplx));
    if (!psi || !hpsi) { free(psi); free(hpsi); return -1; }
    memcpy(psi, psi0, d * sizeof(cplx));
    double lq = 0.0;
    int saved = 0;
    for (int k = 0; k < n_steps; ++k) {
        if (k % save_every == 0) memcpy(shells + (uint64_t)saved++ * d, psi, d * sizeof(cplx));
        orc_hv(n_sites, n_bonds, bonds, K, J, psi, hpsi);
        double uk = creal(dotc(d, psi, hpsi)) / n;
        double q2 = 0.0;
        for (uint64_t x = 0; x < d; ++x) {
            hpsi[x] = ell * psi[x] - hpsi[x] / n;       /* (l - h) psi */
            q2 += creal(hpsi[x]) * creal(hpsi[x]) + cimag(hpsi[x]) * cimag(hpsi[x]);
        }
        double q = sqrt(q2);
        u[k] = uk;
        logQ[k] = lq;
        h2[k] = n * n * (q2 - ell * ell + 2.0 * ell * uk);
        lq += log(q);
        for (uint64_t x = 0; x < d; ++x) psi[x] = hpsi[x] / q;
    }
    free(psi); free(hpsi);
    return saved;
}

/*
 * Dynamical structure factor probe (Sec. V, definition of S^alpha_{+Q}):
 *   lambda = N^{-1/2} sum_l exp(+i Q.R_l) S^gamma_l psi
 * with R_l the real-space position of site l. out_y = sum_l f_l <y|S^g_l|x> psi_x
 * with x = y (gamma = z) or x = y ^ 2^l (gamma = x, y); the matrix element is
 * obtained by acting on the source |x>. Parallel over y.
 */
void orc_apply_op(int n_sites, const double *pos, int gamma, const double *q,
                  const cplx *psi, cplx *out)
{
    int64_t d = (int64_t)1 << n_sites;
    double norm = 1.0 / sqrt((double)n_sites);
    cplx *f = malloc(n_sites * sizeof(cplx));
    for (int l = 0; l < n_sites; ++l)
        f[l] = norm * cexp(I * (q[0] * pos[2 * l] + q[1] * pos[2 * l + 1]));
    #pragma omp parallel for schedule(static)
    for (int64_t y = 0; y < d; ++y) {
        cplx acc = 0;
        for (int l = 0; l < n_sites; ++l) {
            uint64_t x = (uint64_t)y ^ (1ull << l);
            if (gamma == 2)      acc += f[l] * 0.5 * spin(y, l) * psi[y];
            else if (gamma == 0) acc += f[l] * 0.5 * psi[x];
            else                 acc += f[l] * (I * 0.5 * spin(x, l)) * psi[x];
        }
        out[y] = acc;
    }
    free(f);
}

/*
 * Shifted COCG for (z_sigma - H) chi = lambda, returning the projected
 * Green's functions G_sigma = <proj|(z_sigma - H)^{-1}|lambda>, proj = lambda
 * unless given (Sec. II.B, Eq. 'linearSQomega' and the shifted Krylov
 * paragraph; proj = A psi, lambda = B psi gives the A != B response of
 * Eq. 'GAB_TPS').
 *
 * H is real symmetric, so z - H is complex symmetric and BiCG with the
 * shadow residual taken as conj(r) reduces to COCG: all inner products of
 * the seed recurrence are the bilinear r^T r, p^T A p.
 * Seed system A = z_seed - H, textbook two-term form:
 *   p_k = r_k + beta_{k-1} p_{k-1},  q_k = A p_k,  alpha_k = rho_k / p_k^T q_k,
 *   r_{k+1} = r_k - alpha_k q_k,     beta_k = rho_{k+1} / rho_k.
 * Shifted systems A + D_sigma (D_sigma = z_sigma - z_seed) have collinear
 * residuals r^sigma_k = r_k / pi^sigma_k (Frommer 2003, cited in Sec. II.B):
 *   pi_{k+1} = (1 + alpha_k D) pi_k + (alpha_k beta_{k-1}/alpha_{k-1}) (pi_k - pi_{k-1})
 *   alpha^s_k = alpha_k pi_k / pi_{k+1},  beta^s_{k-1} = (pi_{k-1}/pi_k)^2 beta_{k-1}
 *   p^s_k = r_k / pi_k + beta^s_{k-1} p^s_{k-1},   x^s_{k+1} = x^s_k + alpha^s_k p^s_k
 * Projected (unprojected == 0): only proj^dagger p^s and G are carried.
 * Unprojected (unprojected != 0): x^s and p^s vectors are carried explicitly
 * and G = proj^dagger x^s at the end (independent check of the projection).
 * A shift whose residual ||r_{k+1}|| / |pi^sigma_{k+1}| has dropped to
 * tol ||lambda|| is frozen (no further updates of its pi, p, G): far from the
 * seed |pi| grows geometrically and would overflow, while its remaining
 * contributions are below the tolerance.
 * Stop after the first iteration k+1 with
 *   max over unfrozen sigma of ||r_{k+1}|| / |pi^sigma_{k+1}| <= tol ||lambda||.
 * Returns 0 converged, 1 not converged, 2 breakdown.
 */
int orc_cocg(int n_sites, int n_bonds, const int32_t *bonds, double K, double J,
             const cplx *lambda, const cplx *proj, double zs_re, double zs_im, int n_shift,
             const cplx *z, double tol, int max_iter, int unprojected,
             cplx *G, int *iters_out, double *resid_out)
{
    /* G(z) = proj^dagger (z - H)^{-1} lambda; proj NULL: proj = lambda
       (A = B). With proj = A psi and lambda = B psi this is the response
       <psi|A^dagger (z - H)^{-1} B|psi> of two different operators. */
    if (!proj) proj = lambda;
    uint64_t d = 1ull << n_sites;
    cplx z_seed = zs_re + I * zs_im;
    cplx *r = malloc(d * sizeof(cplx)), *p = calloc(d, sizeof(cplx));
    cplx *hp = malloc(d * sizeof(cplx)), *qv = malloc(d * sizeof(cplx));
    cplx *pi_prev = malloc(n_shift * sizeof(cplx)), *pi_cur = malloc(n_shift * sizeof(cplx));
    cplx *pt = calloc(n_shift, sizeof(cplx)), *beta_s = calloc(n_shift, sizeof(cplx));
    char *frozen = calloc(n_shift, 1);
    cplx *xs = NULL, *ps = NULL;
    if (unprojected) {
        xs = calloc((size_t)n_shift * d, sizeof(cplx));
        ps = calloc((size_t)n_shift * d, sizeof(cplx));
    }
    int status = 1, k = 0;
    memcpy(r, lambda, d * sizeof(cplx));
    double lnorm = sqrt(creal(dotc(d, lambda, lambda)));
    for (int s = 0; s < n_shift; ++s) { pi_prev[s] = 1; pi_cur[s] = 1; G[s] = 0; }
    cplx rho = dotu(d, r, r), rho_prev = 1, alpha_prev = 1, beta_prev = 0;
    double worst = 0;
    for (k = 0; k < max_iter; ++k) {
        cplx beta = (k == 0) ? 0 : rho / rho_prev;
        for (uint64_t x = 0; x < d; ++x) p[x] = r[x] + beta * p[x];
        orc_hv(n_sites, n_bonds, bonds, K, J, p, hp);
        for (uint64_t x = 0; x < d; ++x) qv[x] = z_seed * p[x] - hp[x];
        cplx pq = dotu(d, p, qv);
        if (cabs(pq) == 0.0 || cabs(rho) == 0.0) { status = 2; break; }
        cplx alpha = rho / pq;
        cplx g = dotc(d, proj, r);                         /* proj^dagger r_k */
        for (int s = 0; s < n_shift; ++s) {
            if (frozen[s]) continue;
            cplx dz = z[s] - z_seed;
            cplx c = (k == 0) ? 0 : alpha * beta / alpha_prev;
            cplx pi_next = (1.0 + alpha * dz) * pi_cur[s] + c * (pi_cur[s] - pi_prev[s]);
            cplx bs = (k == 0) ? 0 : (pi_prev[s] / pi_cur[s]) * (pi_prev[s] / pi_cur[s]) * beta;
            cplx as = alpha * pi_cur[s] / pi_next;
            if (unprojected) {
                cplx *pv = ps + (size_t)s * d, *xv = xs + (size_t)s * d;
                for (uint64_t x = 0; x < d; ++x) {
                    pv[x] = r[x] / pi_cur[s] + bs * pv[x];
                    xv[x] += as * pv[x];
                }
            } else {
                pt[s] = g / pi_cur[s] + bs * pt[s];
                G[s] += as * pt[s];
            }
            beta_s[s] = bs;
            pi_prev[s] = pi_cur[s];
            pi_cur[s] = pi_next;
        }
        for (uint64_t x = 0; x < d; ++x) r[x] -= alpha * qv[x];
        rho_prev = rho;
        rho = dotu(d, r, r);
        alpha_prev = alpha;
        beta_prev = beta;
        double rn = sqrt(creal(dotc(d, r, r)));
        worst = 0;
        for (int s = 0; s < n_shift; ++s) {
            if (frozen[s]) continue;
            double rs = rn / cabs(pi_cur[s]);
            if (rs <= tol * lnorm) frozen[s] = 1;
            if (rs > worst) worst = rs;
        }
        if (worst <= tol * lnorm) { status = 0; ++k; break; }
    }
    (void)beta_prev;
    if (unprojected) {
        for (int s = 0; s < n_shift; ++s) G[s] = dotc(d, proj, xs + (size_t)s * d);
    }
    *iters_out = k;
    *resid_out = worst / (lnorm > 0 ? lnorm : 1.0);
    free(r); free(p); free(hp); free(qv); free(pi_prev); free(pi_cur); free(pt);
    free(beta_s); free(xs); free(ps); free(frozen);
    return status;
}

/*
 * Canonical ensemble spectrum (Sec. III, Eq. 'chiAB' with A = B = S_q):
 *   S(w, T) = sum_{n,m} exp(-(E_n - E_0)/T) / Z |<m|S_q|n>|^2 (eta/pi) / ((w - (E_m - E_n))^2 + eta^2)
 * a2[n * D + m] = |<m|S_q|n>|^2, E ascending. Parallel over the frequency.
 */
void orc_canonical_dsf(int64_t dim, const double *E, const double *a2,
                       int n_w, const double *w, double eta,
                       int n_T, const double *T, double *S)
{
    for (int t = 0; t < n_T; ++t) {
        double *p = malloc(dim * sizeof(double));
        double z = 0;
        for (int64_t n = 0; n < dim; ++n) { p[n] = exp(-(E[n] - E[0]) / T[t]); z += p[n]; }
        for (int64_t n = 0; n < dim; ++n) p[n] /= z;
        #pragma omp parallel for schedule(static)
        for (int iw = 0; iw < n_w; ++iw) {
            double acc = 0;
            for (int64_t n = 0; n < dim; ++n) {
                if (p[n] < 1e-300) continue;
                double part = 0;
                for (int64_t m = 0; m < dim; ++m) {
                    double a = a2[n * dim + m];
                    if (a == 0.0) continue;
                    double dw = w[iw] - (E[m] - E[n]);
                    part += a * (eta / ORC_PI) / (dw * dw + eta * eta);
                }
                acc += p[n] * part;
            }
            S[(int64_t)t * n_w + iw] = acc;
        }
        free(p);
    }
}

/* ---------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11 "Parallel random numbers:
 * as easy as 1, 2, 3"), written from its published definition:
 * one round maps (c0,c1,c2,c3) with key (k0,k1) to
 *   (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0)),
 * M0 = 0xD2511F53, M1 = 0xCD9E8D57; the key is bumped by
 * (0x9E3779B9, 0xBB67AE85) between rounds; 10 rounds.
 * ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t *ctr_in, const uint32_t *key_in, uint32_t *out)
{
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
    memcpy(out, c, sizeof c);
}

/*
 * Random initial TPQ vector (Sec. II.A): c_x complex Gaussian, normalised,
 * so the state is uniform on the unit sphere of R^{2 N_F}.
 * Element x draws one Philox block with counter (x_lo, x_hi, sample, 0) and
 * key (seed_lo, seed_hi); u1 = (w0:w1 >> 11 + 0.5) 2^-53, u2 = (w2:w3 >> 11 + 0.5) 2^-53;
 * Box-Muller: c_x = sqrt(-2 ln u1) (cos 2 pi u2 + i sin 2 pi u2).
 */
void orc_gaussian_state(int n_sites, uint64_t seed, uint32_t sample, cplx *out)
{
    uint64_t d = 1ull << n_sites;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    double nrm = 0;
    for (uint64_t x = 0; x < d; ++x) {
        uint32_t ctr[4] = {(uint32_t)x, (uint32_t)(x >> 32), sample, 0}, w[4];
        orc_philox4x32_10(ctr, key, w);
        double u1 = ((double)((((uint64_t)w[0] << 32) | w[1]) >> 11) + 0.5) * 0x1p-53;
        double u2 = ((double)((((uint64_t)w[2] << 32) | w[3]) >> 11) + 0.5) * 0x1p-53;
        double rad = sqrt(-2.0 * log(u1));
        out[x] = rad * cos(2.0 * ORC_PI * u2) + I * rad * sin(2.0 * ORC_PI * u2);
        nrm += rad * rad;
    }
    nrm = sqrt(nrm);
    for (uint64_t x = 0; x < d; ++x) out[x] /= nrm;
}
