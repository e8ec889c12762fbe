/*
 * oracle.c -- plain, slow, FP64 CPU oracle for the muon-tomography
 * log-posterior of layered block-cave geometries and its Metropolis update.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / --impl reference legs use it.  It shares no source with the
 * CUDA library (own Philox, own geometry, own march, own sampler).
 *
 * Every routine follows the paper ("GPU-accelerated Bayesian inference for
 * block-cave geometry recovery via muon tomography") step by step, in FP64,
 * with no blocking, fusion or reordering beyond what the cited definition
 * states.  Readings of points the paper leaves open are marked READING.
 *
 * Conventions (READING, the paper fixes none of these):
 *   box [0,Lx]x[0,Ly]x[0,Lz]; heights are z above the box floor (Sec. 2.1.3,
 *   "relative height with respect to the floor"); heights[l][r][c] row-major,
 *   right-most index fastest (Fig. "array_indexing"); surface nodes sit on
 *   the grid corners x_c = c*Lx/(Q-1), y_r = r*Ly/(R-1) and are interpolated
 *   bilinearly; surfaces l = 0..L-1 bottom to top, units u = 0..L with unit u
 *   between surface u-1 (below) and surface u (above).
 *
 * Parity pins: see tests/test_oracle_*.py.  Every function below is pinned
 * by at least one closed form, invariant, library routine or brute force.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int L, R, Q;            /* surfaces, rows (y), cols (x) */
    double box[3];          /* Lx, Ly, Lz in metres */
    const double *rho;      /* [L+1] unit densities bottom->top, g/cc */
    int S, P;               /* sensors, pixels per sensor */
    const double *sensor;   /* [S][3] sensor positions (inside the box) */
    const double *dir;      /* [P][3] unit pixel directions, shared by sensors */
    const int32_t *counts;  /* [S][P] observed counts (may be NULL) */
    int G;                  /* samples per ray */
    double gamma;           /* sigmoid scale (m); 0 = Heaviside */
    double I0, Lambda;      /* flux model lambda = I0 exp(-O/Lambda) */
    double tau, car_r, delta; /* prior: precision scale, CAR r, min thickness */
    const double *mu;       /* [L][R][Q] prior mean */
} or_problem;

/* ------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11).  The paper draws its random numbers inside
 * NumPyro; this counter-based generator is READING: counter = {index, step,
 * chain, stream}, key = {seed lo, seed hi}.
 * ---------------------------------------------------------------------- */
void or_philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;  /* Weyl key schedule */
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Stream identifiers (READING). */
enum { OR_GEOM = 0, OR_DATA = 1, OR_INIT = 2, OR_PROP = 3, OR_ACC = 4, OR_MALA = 5 };

static void draw(uint64_t seed, uint32_t stream, uint32_t chain, uint32_t step,
                 uint32_t index, uint32_t w[4])
{
    uint32_t ctr[4] = {index, step, chain, stream};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    or_philox(ctr, key, w);
}

/* Uniform on (0,1): u = (floor(r64 / 2^12) + 1/2) * 2^-52 with r64 = hi:lo.
 * The numerator has at most 53 significant bits, so u is exact in FP64. */
double or_u01(uint32_t lo, uint32_t hi)
{
    uint64_t r = ((uint64_t)hi << 32) | (uint64_t)lo;
    return ((double)(r >> 12) + 0.5) * 0x1p-52;
}

/* Box-Muller: normals 2j and 2j+1 come from counter index j. */
void or_normals(uint64_t seed, uint32_t stream, uint32_t chain, uint32_t step,
                int n, double *z)
{
    const double two_pi = 6.283185307179586476925286766559;
    for (int i = 0; i < n; i += 2) {
        uint32_t w[4];
        draw(seed, stream, chain, step, (uint32_t)(i / 2), w);
        double u1 = or_u01(w[0], w[1]);
        double u2 = or_u01(w[2], w[3]);
        double rad = sqrt(-2.0 * log(u1));
        z[i] = rad * cos(two_pi * u2);
        if (i + 1 < n) z[i + 1] = rad * sin(two_pi * u2);
    }
}

/* ------------------------------------------------------------------------
 * Geometry.
 * ---------------------------------------------------------------------- */

/* Distance from o (inside the box) along d to the box boundary: the ray
 * starts at the sensor (Sec. 2.1.1, opacity integral) and only the part
 * inside the domain D contributes (READING: rho is defined on D only). */
double or_t_exit(const double o[3], const double d[3], const double box[3])
{
    double t = INFINITY;
    for (int a = 0; a < 3; ++a) {
        double ta = INFINITY;
        if (d[a] > 0.0) ta = (box[a] - o[a]) / d[a];
        else if (d[a] < 0.0) ta = (0.0 - o[a]) / d[a];
        if (ta < t) t = ta;
    }
    return t;
}

/* Height of one surface at (x, y): bilinear interpolation of the node
 * heights H_{l,x,y} (Sec. 2.1.3, layer model on an n_rows x n_cols grid;
 * the interpolant between nodes is READING). */
double or_surface(int R, int Q, const double box[3], const double *h, double x, double y)
{
    double gx = x / box[0] * (double)(Q - 1);
    double gy = y / box[1] * (double)(R - 1);
    if (gx < 0.0) gx = 0.0;
    if (gx > (double)(Q - 1)) gx = (double)(Q - 1);
    if (gy < 0.0) gy = 0.0;
    if (gy > (double)(R - 1)) gy = (double)(R - 1);
    int c0 = (int)floor(gx), r0 = (int)floor(gy);
    if (c0 > Q - 2) c0 = Q - 2;
    if (r0 > R - 2) r0 = R - 2;
    double tx = gx - (double)c0, ty = gy - (double)r0;
    double h00 = h[r0 * Q + c0], h01 = h[r0 * Q + c0 + 1];
    double h10 = h[(r0 + 1) * Q + c0], h11 = h[(r0 + 1) * Q + c0 + 1];
    return (1.0 - tx) * (1.0 - ty) * h00 + tx * (1.0 - ty) * h01
         + (1.0 - tx) * ty * h10 + tx * ty * h11;
}

/* Scaled sigmoid varsigma_gamma(u) = 1 / (1 + exp(-u/gamma)) (Eq.
 * def_sigmoid); gamma = 0 selects the Heaviside eta with eta(0) = 1/2
 * (Sec. 2.1.4, definition of eta). */
double or_sigma(double u, double gamma)
{
    if (gamma == 0.0) {
        if (u < 0.0) return 0.0;
        if (u == 0.0) return 0.5;
        return 1.0;
    }
    return 1.0 / (1.0 + exp(-u / gamma));
}

/* Opacity of one ray through the geometry H[L][R][Q] (Sec. 2.1.1, opacity
 * O = integral of rho along the ray), evaluated as a midpoint sum over G
 * samples t_k = (k + 1/2) dt, dt = t_exit / G.  At each sample the density
 * is the normalised smooth-indicator mixture R_hat = sum_u W_u rho_u with
 * D_u = varsigma(s_u - z) - varsigma(s_{u-1} - z), W_u = D_u / sum D (Eqs.
 * smooth_layer_indicators and def_LM_density_grid_smooth); the bottom and
 * top units use varsigma(-inf) = 0 and varsigma(+inf) = 1 (READING).
 * unit_len (nullable, [L+1]) receives the path length per unit,
 * dt * sum_k W_u(k).  Returns O in g/cc * m (= metres water equivalent). */
double or_ray_opacity(const or_problem *pb, const double *H, int s, int p, double *unit_len)
{
    const int L = pb->L;
    const double *o = pb->sensor + 3 * s;
    const double *d = pb->dir + 3 * p;
    double te = or_t_exit(o, d, pb->box);
    double dt = te / (double)pb->G;
    double sig[L + 2];
    double len[L + 1];
    for (int u = 0; u <= L; ++u) len[u] = 0.0;
    double O = 0.0;
    for (int k = 0; k < pb->G; ++k) {
        double t = ((double)k + 0.5) * dt;
        double x = o[0] + t * d[0], y = o[1] + t * d[1], z = o[2] + t * d[2];
        /* sig[l+1] = varsigma(s_l - z); sig[0] = 0 below, sig[L+1] = 1 above */
        sig[0] = 0.0;
        for (int l = 0; l < L; ++l) {
            double sl = or_surface(pb->R, pb->Q, pb->box, H + (size_t)l * pb->R * pb->Q, x, y);
            sig[l + 1] = or_sigma(sl - z, pb->gamma);
        }
        sig[L + 1] = 1.0;
        double Dsum = 0.0;
        double D[L + 1];
        for (int u = 0; u <= L; ++u) {
            D[u] = sig[u + 1] - sig[u];
            Dsum += D[u];
        }
        double rho_hat = 0.0;
        for (int u = 0; u <= L; ++u) {
            double W = D[u] / Dsum;
            rho_hat += W * pb->rho[u];
            len[u] += W;
        }
        O += rho_hat;
    }
    if (unit_len)
        for (int u = 0; u <= L; ++u) unit_len[u] = len[u] * dt;
    return O * dt;
}

/* Expected count lambda = I0 exp(-O / Lambda): the flux model that stands
 * in for Eq. expected_counts (intensity times efficiency over the pixel's
 * solid angle, which the paper does not give). */
double or_lambda(double O, double I0, double Lambda)
{
    return I0 * exp(-O / Lambda);
}

/* Poisson log-pmf, C ln(lambda) - lambda - ln C! (Eq. def_likelihood). */
double or_poisson_logpmf(int32_t C, double lam)
{
    if (C == 0) return -lam;
    return (double)C * log(lam) - lam - lgamma((double)C + 1.0);
}

/* The same term in centred form: with y = ln(I0/C) - O/Lambda (so that
 * lambda = C e^y) it equals K + C y - C expm1(y), K = C ln C - C - ln C!.
 * The algebra is exact; this form avoids cancelling two large numbers. */
double or_poisson_logpmf_centred(int32_t C, double O, double I0, double Lambda)
{
    if (C == 0) return -I0 * exp(-O / Lambda);
    double c = (double)C;
    double K = c * log(c) - c - lgamma(c + 1.0);
    double y = log(I0 / c) - O / Lambda;
    return K + c * y - c * expm1(y);
}

/* Log-likelihood of one geometry: sum over sensors and pixels of the
 * Poisson terms, pixels conditionally independent (Eq. def_likelihood). */
double or_loglik(const or_problem *pb, const double *H)
{
    double ll = 0.0;
    for (int s = 0; s < pb->S; ++s)
        for (int p = 0; p < pb->P; ++p) {
            double O = or_ray_opacity(pb, H, s, p, NULL);
            double lam = or_lambda(O, pb->I0, pb->Lambda);
            ll += or_poisson_logpmf(pb->counts[(size_t)s * pb->P + p], lam);
        }
    return ll;
}

/* Per-ray terms of one geometry, [S][P] (for element-wise parity). */
void or_loglik_terms(const or_problem *pb, const double *H, double *terms, double *opacity)
{
    for (int s = 0; s < pb->S; ++s)
        for (int p = 0; p < pb->P; ++p) {
            double O = or_ray_opacity(pb, H, s, p, NULL);
            size_t i = (size_t)s * pb->P + p;
            if (opacity) opacity[i] = O;
            if (terms) terms[i] = or_poisson_logpmf(pb->counts[i], or_lambda(O, pb->I0, pb->Lambda));
        }
}

/* Log-prior (unnormalised).  Ordering and bounds: every thickness at least
 * delta ("strictly positive thicknesses", Sec. 2.1.3) and 0 <= H <= Lz,
 * else -inf.  Smoothness: the CAR precision Q = diag(A 1) - r A on the
 * periodic nearest-neighbour grid (Eq. def_CAR_precision, Fig. neighbors),
 * used as a Gaussian quadratic form -tau/2 (h_l - mu_l)^T Q (h_l - mu_l) on
 * each surface's heights (READING: the paper puts Q inside a copula prior).
 * On a periodic grid every node has 4 neighbours, so (A 1)_i = 4; for a
 * side of length 2 the two wrap-around neighbours coincide and count twice. */
double or_logprior(const or_problem *pb, const double *H)
{
    const int L = pb->L, R = pb->R, Q = pb->Q;
    const size_t N = (size_t)R * Q;
    for (int l = 0; l < L; ++l)
        for (size_t i = 0; i < N; ++i) {
            double h = H[l * N + i];
            if (!(h >= 0.0 && h <= pb->box[2])) return -INFINITY;
            if (l > 0 && !(h - H[(l - 1) * N + i] >= pb->delta)) return -INFINITY;
        }
    double quad = 0.0;
    for (int l = 0; l < L; ++l) {
        const double *h = H + l * N, *m = pb->mu + l * N;
        for (int r = 0; r < R; ++r)
            for (int c = 0; c < Q; ++c) {
                int up = (r + 1) % R, dn = (r + R - 1) % R;
                int rt = (c + 1) % Q, lf = (c + Q - 1) % Q;
                double e = h[r * Q + c] - m[r * Q + c];
                double nb = (h[up * Q + c] - m[up * Q + c]) + (h[dn * Q + c] - m[dn * Q + c])
                          + (h[r * Q + rt] - m[r * Q + rt]) + (h[r * Q + lf] - m[r * Q + lf]);
                quad += e * (4.0 * e - pb->car_r * nb);
            }
    }
    return -0.5 * pb->tau * quad;
}

/* ------------------------------------------------------------------------
 * Synthetic observed counts: C_p ~ Poisson(lambda_p(H_true)) (Eq.
 * def_likelihood); the paper rounds lambda instead (Sec. 4), kept as
 * count_mode 1.  Draws use stream DATA with counter {ray, attempt, 0}.
 * ---------------------------------------------------------------------- */

/* Knuth's multiplication method (lambda < 10) and Hormann's transformed
 * rejection with squeeze, PTRS (W. Hormann, "The transformed rejection
 * method for generating Poisson random variables", Insurance: Mathematics
 * and Economics 12, 1993) for lambda >= 10.  Attempts are bounded; running
 * out sets *status = 1. */
static int32_t poisson_draw_n(double lam, uint64_t seed, uint32_t ray, int *status, int *attempts)
{
    const int max_attempts = 256;
    if (lam < 10.0) {
        double limit = exp(-lam);
        double prod = 1.0;
        int32_t k = 0;
        for (int j = 0; j < max_attempts; ++j) {
            uint32_t w[4];
            draw(seed, OR_DATA, 0, (uint32_t)j, ray, w);
            double uu[2] = {or_u01(w[0], w[1]), or_u01(w[2], w[3])};
            for (int h = 0; h < 2; ++h) {
                prod = prod * uu[h];
                if (prod <= limit) {
                    if (attempts) *attempts = j + 1;
                    return k;
                }
                k = k + 1;
            }
        }
        if (status) *status = 1;
        if (attempts) *attempts = max_attempts;
        return k;
    }
    double slam = sqrt(lam);
    double loglam = log(lam);
    double b = 0.931 + 2.53 * slam;
    double a = -0.059 + 0.02483 * b;
    double inv_alpha = 1.1239 + 1.1328 / (b - 3.4);
    double v_r = 0.9277 - 3.6224 / (b - 2.0);
    for (int j = 0; j < max_attempts; ++j) {
        uint32_t w[4];
        draw(seed, OR_DATA, 0, (uint32_t)j, ray, w);
        double U = or_u01(w[0], w[1]) - 0.5;
        double V = or_u01(w[2], w[3]);
        double us = 0.5 - fabs(U);
        double kf = floor((2.0 * a / us + b) * U + lam + 0.43);
        if (attempts) *attempts = j + 1;
        if (us >= 0.07 && V <= v_r) return (int32_t)kf;
        if (kf < 0.0 || (us < 0.013 && V > us)) continue;
        double lhs = log(V) + log(inv_alpha) - log(a / (us * us) + b);
        double rhs = -lam + kf * loglam - lgamma(kf + 1.0);
        if (lhs <= rhs) return (int32_t)kf;
    }
    if (status) *status = 1;
    if (attempts) *attempts = max_attempts;
    return 0;
}

int32_t or_poisson_draw(double lam, uint64_t seed, uint32_t ray, int *status)
{
    return poisson_draw_n(lam, seed, ray, status, NULL);
}

/* Test instrumentation (no arithmetic of its own): the mean number of
 * attempts or_poisson_draw takes for lambda over rays 0 .. n-1.  For
 * lambda >= 10 one attempt of the transformed rejection accepts value k with
 * probability p(k) / inv_alpha (the hat dominates p), so the attempts are
 * geometric with mean inv_alpha = 1.1239 + 1.1328 / (b - 3.4). */
double or_poisson_mean_attempts(double lam, uint64_t seed, int n)
{
    double tot = 0.0;
    for (int i = 0; i < n; ++i) {
        int att = 0, st = 0;
        poisson_draw_n(lam, seed, (uint32_t)i, &st, &att);
        tot += att;
    }
    return n > 0 ? tot / n : 0.0;
}

/* Counts for every (sensor, pixel) of the true geometry; lambda_out and
 * counts_out are [S][P].  count_mode 0 = Poisson draw, 1 = round half to
 * even (Sec. 4, expected counts rounded to the nearest integer).  Returns
 * the number of draws that ran out of attempts. */
int or_generate_counts(const or_problem *pb, const double *H_true, uint64_t seed,
                       int count_mode, int32_t *counts_out, double *lambda_out)
{
    int bad = 0;
    for (int s = 0; s < pb->S; ++s)
        for (int p = 0; p < pb->P; ++p) {
            size_t i = (size_t)s * pb->P + p;
            double lam = or_lambda(or_ray_opacity(pb, H_true, s, p, NULL), pb->I0, pb->Lambda);
            if (lambda_out) lambda_out[i] = lam;
            int st = 0;
            int32_t c = count_mode == 1 ? (int32_t)nearbyint(lam)
                                        : or_poisson_draw(lam, seed, (uint32_t)i, &st);
            bad += st;
            if (counts_out) counts_out[i] = c;
        }
    return bad;
}

/* ------------------------------------------------------------------------
 * Metropolis-Hastings (Sec. 2.2: MCMC needs only ratios of the posterior
 * density).  Random-walk proposal H' = H + sigma * xi, xi ~ N(0, I) from
 * stream PROP, counter {j, step, chain}; acceptance uniform from stream ACC,
 * counter {0, step, chain}.
 * ---------------------------------------------------------------------- */
void or_rw_propose(const or_problem *pb, const double *H, double sigma, uint64_t seed,
                   uint32_t chain, uint32_t step, double *H_prop)
{
    int n = pb->L * pb->R * pb->Q;
    double *xi = (double *)malloc(sizeof(double) * (size_t)n);
    or_normals(seed, OR_PROP, chain, step, n, xi);
    for (int i = 0; i < n; ++i) H_prop[i] = H[i] + sigma * xi[i];
    free(xi);
}

double or_accept_logu(uint64_t seed, uint32_t chain, uint32_t step)
{
    uint32_t w[4];
    draw(seed, OR_ACC, chain, step, 0, w);
    return log(or_u01(w[0], w[1]));
}

/* Accept iff the proposal has finite prior and ln u < (new) - (old). */
int or_mh_decide(double lp_new, double ll_new, double lp_old, double ll_old, double logu)
{
    if (!(lp_new > -INFINITY)) return 0;
    double delta = (ll_new + lp_new) - (ll_old + lp_old);
    return logu < delta;
}

/* n_steps of random-walk Metropolis for one chain, in place.  Steps are
 * numbered step0 .. step0+n_steps-1.  use_lik = 0 targets the prior alone.
 * Returns the number of accepted proposals; lp/ll hold the final state's. */
int or_rw_chain(const or_problem *pb, double *H, double sigma, uint64_t seed, uint32_t chain,
                uint32_t step0, int n_steps, int use_lik, double *lp_io, double *ll_io,
                double *trace /* nullable [n_steps][L*R*Q] */)
{
    int n = pb->L * pb->R * pb->Q;
    double *Hp = (double *)malloc(sizeof(double) * (size_t)n);
    double lp = or_logprior(pb, H);
    double ll = use_lik ? or_loglik(pb, H) : 0.0;
    int acc = 0;
    for (int it = 0; it < n_steps; ++it) {
        uint32_t step = step0 + (uint32_t)it;
        or_rw_propose(pb, H, sigma, seed, chain, step, Hp);
        double lpn = or_logprior(pb, Hp);
        double lln = (use_lik && lpn > -INFINITY) ? or_loglik(pb, Hp) : 0.0;
        if (or_mh_decide(lpn, lln, lp, ll, or_accept_logu(seed, chain, step))) {
            memcpy(H, Hp, sizeof(double) * (size_t)n);
            lp = lpn;
            ll = lln;
            ++acc;
        }
        if (trace) memcpy(trace + (size_t)it * n, H, sizeof(double) * (size_t)n);
    }
    free(Hp);
    if (lp_io) *lp_io = lp;
    if (ll_io) *ll_io = ll;
    return acc;
}

/* ------------------------------------------------------------------------
 * Gradient of the log-posterior with respect to every node height (the
 * differentiable forward model the paper builds for gradient-based
 * samplers, Sec. 2.1.4).  Analytic reverse of or_ray_opacity:
 *   d ll / d O_p = (lambda_p - C_p) / Lambda,
 *   d O_p / d h_{l,n} = dt * sum_k (rho_l - rho_{l+1}) varsigma'(s_l - z_k) w_n(x_k),
 * with varsigma' = varsigma (1 - varsigma) / gamma and w_n the bilinear
 * weight of node n (the normaliser sum D is identically 1, so W = D has the
 * same derivative), and d lp / d h_l = -tau Q (h_l - mu_l).  gamma > 0 only.
 * ---------------------------------------------------------------------- */
static void add_bilinear_grad(int R, int Q, const double box[3], double *g, double x, double y,
                              double v)
{
    double gx = x / box[0] * (double)(Q - 1);
    double gy = y / box[1] * (double)(R - 1);
    if (gx < 0.0) gx = 0.0;
    if (gx > (double)(Q - 1)) gx = (double)(Q - 1);
    if (gy < 0.0) gy = 0.0;
    if (gy > (double)(R - 1)) gy = (double)(R - 1);
    int c0 = (int)floor(gx), r0 = (int)floor(gy);
    if (c0 > Q - 2) c0 = Q - 2;
    if (r0 > R - 2) r0 = R - 2;
    double tx = gx - (double)c0, ty = gy - (double)r0;
    g[r0 * Q + c0] += v * (1.0 - tx) * (1.0 - ty);
    g[r0 * Q + c0 + 1] += v * tx * (1.0 - ty);
    g[(r0 + 1) * Q + c0] += v * (1.0 - tx) * ty;
    g[(r0 + 1) * Q + c0 + 1] += v * tx * ty;
}

void or_grad_loglik(const or_problem *pb, const double *H, double *grad /* [L][R][Q] */)
{
    const int L = pb->L;
    const size_t N = (size_t)pb->R * pb->Q;
    memset(grad, 0, sizeof(double) * L * N);
    for (int s = 0; s < pb->S; ++s)
        for (int p = 0; p < pb->P; ++p) {
            size_t i = (size_t)s * pb->P + p;
            double O = or_ray_opacity(pb, H, s, p, NULL);
            double lam = or_lambda(O, pb->I0, pb->Lambda);
            double dO = (lam - (double)pb->counts[i]) / pb->Lambda;
            const double *o = pb->sensor + 3 * s, *d = pb->dir + 3 * p;
            double dt = or_t_exit(o, d, pb->box) / (double)pb->G;
            for (int k = 0; k < pb->G; ++k) {
                double t = ((double)k + 0.5) * dt;
                double x = o[0] + t * d[0], y = o[1] + t * d[1], z = o[2] + t * d[2];
                for (int l = 0; l < L; ++l) {
                    double sl = or_surface(pb->R, pb->Q, pb->box, H + l * N, x, y);
                    double sg = or_sigma(sl - z, pb->gamma);
                    double dsig = sg * (1.0 - sg) / pb->gamma;
                    double v = dO * dt * (pb->rho[l] - pb->rho[l + 1]) * dsig;
                    add_bilinear_grad(pb->R, pb->Q, pb->box, grad + l * N, x, y, v);
                }
            }
        }
}

void or_grad_logprior(const or_problem *pb, const double *H, double *grad)
{
    const int R = pb->R, Q = pb->Q;
    const size_t N = (size_t)R * Q;
    for (int l = 0; l < pb->L; ++l) {
        const double *h = H + l * N, *m = pb->mu + l * N;
        for (int r = 0; r < R; ++r)
            for (int c = 0; c < Q; ++c) {
                int up = (r + 1) % R, dn = (r + R - 1) % R;
                int rt = (c + 1) % Q, lf = (c + Q - 1) % Q;
                double e = h[r * Q + c] - m[r * Q + c];
                double nb = (h[up * Q + c] - m[up * Q + c]) + (h[dn * Q + c] - m[dn * Q + c])
                          + (h[r * Q + rt] - m[r * Q + rt]) + (h[r * Q + lf] - m[r * Q + lf]);
                grad[l * N + r * Q + c] = -pb->tau * (4.0 * e - pb->car_r * nb);
            }
    }
}

/* ------------------------------------------------------------------------
 * MALA (Metropolis-adjusted Langevin): H' = H + (eps^2/2) grad + eps xi with
 * xi from stream MALA, accepted with the Hastings correction
 * ln q(H | H') - ln q(H' | H), q(b | a) = N(b; a + (eps^2/2) grad(a), eps^2 I).
 * ---------------------------------------------------------------------- */
void or_mala_propose(const or_problem *pb, const double *H, const double *grad, double eps,
                     uint64_t seed, uint32_t chain, uint32_t step, double *H_prop)
{
    int n = pb->L * pb->R * pb->Q;
    double *xi = (double *)malloc(sizeof(double) * (size_t)n);
    or_normals(seed, OR_MALA, chain, step, n, xi);
    for (int i = 0; i < n; ++i) H_prop[i] = H[i] + 0.5 * eps * eps * grad[i] + eps * xi[i];
    free(xi);
}

/* ln q(b | a) up to the constant shared by both directions. */
double or_mala_logq(int n, const double *b, const double *a, const double *grad_a, double eps)
{
    double ss = 0.0;
    for (int i = 0; i < n; ++i) {
        double r = b[i] - a[i] - 0.5 * eps * eps * grad_a[i];
        ss += r * r;
    }
    return -ss / (2.0 * eps * eps);
}

/* ------------------------------------------------------------------------
 * Batch log-likelihood over chains, threaded over (chain, sensor) items.
 * Used to time the oracle on the host; the arithmetic is or_loglik's.
 * ---------------------------------------------------------------------- */
typedef struct {
    const or_problem *pb;
    const double *H;
    int n_chains;
    double *partial;          /* [n_chains][S] */
    int next, stride;         /* static round-robin */
} batch_job;

typedef struct { batch_job *job; int tid; } batch_arg;

static void *batch_worker(void *arg_)
{
    batch_arg *arg = (batch_arg *)arg_;
    batch_job *job = arg->job;
    const or_problem *pb = job->pb;
    size_t per_chain = (size_t)pb->L * pb->R * pb->Q;
    int items = job->n_chains * pb->S;
    for (int it = arg->tid; it < items; it += job->stride) {
        int c = it / pb->S, s = it % pb->S;
        const double *H = job->H + (size_t)c * per_chain;
        double acc = 0.0;
        for (int p = 0; p < pb->P; ++p) {
            double O = or_ray_opacity(pb, H, s, p, NULL);
            acc += or_poisson_logpmf(pb->counts[(size_t)s * pb->P + p],
                                     or_lambda(O, pb->I0, pb->Lambda));
        }
        job->partial[it] = acc;
    }
    return NULL;
}

void or_loglik_batch(const or_problem *pb, int n_chains, const double *H, double *out, int n_threads)
{
    if (n_threads < 1) n_threads = 1;
    batch_job job = {pb, H, n_chains, NULL, 0, n_threads};
    job.partial = (double *)malloc(sizeof(double) * (size_t)n_chains * pb->S);
    pthread_t th[n_threads];
    batch_arg args[n_threads];
    for (int t = 0; t < n_threads; ++t) {
        args[t].job = &job;
        args[t].tid = t;
        pthread_create(&th[t], NULL, batch_worker, &args[t]);
    }
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
    for (int c = 0; c < n_chains; ++c) {
        double acc = 0.0;
        for (int s = 0; s < pb->S; ++s) acc += job.partial[(size_t)c * pb->S + s];
        out[c] = acc;
    }
    free(job.partial);
}
