/*
 * tvspec_oracle.c -- plain FP64 CPU oracle of the classical spectral total-variation
 * decomposition (arXiv 2006.10004, Sec. 2.1-2.2).
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the benchmark's CPU-baseline leg
 * load this library. The product path (the CUDA library under paper_2006_10004_gb300/) never
 * links, imports or calls it, and it shares no code with that path.
 *
 * What it computes, step by step, in the paper's notation:
 *   - the TV flow u_t = -p, p in dJ_TV(u), u(0) = f                         (Eq. TVflow)
 *   - discretised by implicit Euler: u(t+dt) = argmin_v 1/2|u(t)-v|^2 + dt J_TV(v)  (Eq. ROF)
 *   - each ROF step solved by a fixed number of Chambolle projection iterations (the
 *     "projection algorithm by Chambolle" of Sec. 4.3, Chambolle 2004) with the isotropic
 *     discrete TV (the Euclidean pointwise norm of Eq. TV);
 *   - the TV transform phi(t) = t u_tt(t)                                     (Eq. TVtrafo)
 *     by a second time difference, its spectrum S(t) = |phi(t)|_L1           (Sec. 2.1)
 *   - band sums b^m = int_{e_m}^{e_{m+1}} phi dt                               (Eq. spectral_bands)
 *   - the residual f_r(T) = u(T) - T u_t(T)                                   (Eq. finite_inverse_trafo)
 *   - filtered images f_H = int_0^T phi(t) H(t) dt + h_r f_r                  (Eq. filteredTVtrafo
 *     substituted into Eq. finite_inverse_trafo; h_r weighs the residual)
 *   - a Parseval-type spectrum <phi(t), f>                                    (Sec. 2.1 names it)
 *
 * Readings of points the paper leaves open:
 *   - forward differences with a zero last row/column (Neumann), divergence = -grad^T;
 *   - K ROF steps give u_0..u_K; phi_k = t_k (u_{k+1} - 2u_k + u_{k-1}) / dt^2 for k=1..K-1,
 *     t_k = k dt; S has K-1 entries;
 *   - band m takes the phi_k with e_m <= t_k < e_{m+1}, Riemann weight dt;
 *   - f_r = u_{K-1} - t_{K-1} (u_K - u_{K-1}) / dt  (the forward difference for u_t(T));
 *   - the dual field p is carried from one ROF step to the next (warm start) unless
 *     warm_start == 0.
 *
 * Everything is double precision and written as plain loops. Loops over pixels that are
 * independent of each other may run on several OpenMP threads; sums over pixels are
 * sequential in row-major order. Compile with -ffp-contract=off so that every expression is
 * evaluated exactly as written.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Images smaller than this run single-threaded (thread start-up would dominate). */
#define OMP_MIN_PIXELS 65536

#define IDX(i, j) ((size_t)(i) * (size_t)W + (size_t)(j))

/* Sets the number of OpenMP threads later calls use (n >= 1); returns the new maximum. */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1)
        omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Discrete gradient (Chambolle 2004, Sec. 2): forward differences,
 *   (grad u)^1_{ij} = u_{i+1,j} - u_{ij} for i < H-1, 0 for i = H-1   (along rows i)
 *   (grad u)^2_{ij} = u_{i,j+1} - u_{ij} for j < W-1, 0 for j = W-1   (along columns j)
 * The zero last row/column is the Neumann boundary condition.
 */
void orc_grad(const double *u, int H, int W, double *g1, double *g2)
{
#pragma omp parallel for schedule(static) if ((size_t)H * (size_t)W >= OMP_MIN_PIXELS)
    for (int i = 0; i < H; ++i) {
        for (int j = 0; j < W; ++j) {
            g1[IDX(i, j)] = (i < H - 1) ? u[IDX(i + 1, j)] - u[IDX(i, j)] : 0.0;
            g2[IDX(i, j)] = (j < W - 1) ? u[IDX(i, j + 1)] - u[IDX(i, j)] : 0.0;
        }
    }
}

/*
 * Discrete divergence, defined as the negative adjoint of orc_grad (Chambolle 2004, Sec. 2):
 *   (div p)_{ij} = a_{ij} + b_{ij},
 *   a_{ij} = [i < H-1] p^1_{ij} - [i > 0] p^1_{i-1,j},
 *   b_{ij} = [j < W-1] p^2_{ij} - [j > 0] p^2_{i,j-1}.
 * The bracket factors drop the terms that the adjoint of the zero last row/column removes.
 */
void orc_div(const double *p1, const double *p2, int H, int W, double *d)
{
#pragma omp parallel for schedule(static) if ((size_t)H * (size_t)W >= OMP_MIN_PIXELS)
    for (int i = 0; i < H; ++i) {
        for (int j = 0; j < W; ++j) {
            double a = (i < H - 1 ? p1[IDX(i, j)] : 0.0) - (i > 0 ? p1[IDX(i - 1, j)] : 0.0);
            double b = (j < W - 1 ? p2[IDX(i, j)] : 0.0) - (j > 0 ? p2[IDX(i, j - 1)] : 0.0);
            d[IDX(i, j)] = a + b;
        }
    }
}

/*
 * n_iter iterations of Chambolle's projection algorithm for one ROF step
 *   u = argmin_v 1/2 |v - g|^2 + lambda J_TV(v)      (Eq. ROF with dt = lambda)
 * One iteration:
 *   w = div p - g / lambda
 *   G = grad w
 *   p <- (p + tau G) / (1 + tau |G|),   |G| = sqrt(G^1^2 + G^2^2) pointwise (isotropic)
 * After the iterations: u = g - lambda div p.
 * p1, p2 hold the starting dual field on entry and the final one on exit.
 * Returns 0, or -1 if scratch memory cannot be allocated.
 */
int orc_chambolle(const double *g, int H, int W, double lambda, double tau, int n_iter,
                  double *p1, double *p2, double *u_out)
{
    size_t N = (size_t)H * (size_t)W;
    double *d = (double *)malloc(N * sizeof(double));
    double *w = (double *)malloc(N * sizeof(double));
    double *G1 = (double *)malloc(N * sizeof(double));
    double *G2 = (double *)malloc(N * sizeof(double));
    if (!d || !w || !G1 || !G2) {
        free(d); free(w); free(G1); free(G2);
        return -1;
    }
    for (int it = 0; it < n_iter; ++it) {
        orc_div(p1, p2, H, W, d);
#pragma omp parallel for schedule(static) if (N >= OMP_MIN_PIXELS)
        for (long long n = 0; n < (long long)N; ++n)
            w[n] = d[n] - g[n] / lambda;
        orc_grad(w, H, W, G1, G2);
#pragma omp parallel for schedule(static) if (N >= OMP_MIN_PIXELS)
        for (long long n = 0; n < (long long)N; ++n) {
            double norm = sqrt(G1[n] * G1[n] + G2[n] * G2[n]);
            double denom = 1.0 + tau * norm;
            p1[n] = (p1[n] + tau * G1[n]) / denom;
            p2[n] = (p2[n] + tau * G2[n]) / denom;
        }
    }
    orc_div(p1, p2, H, W, d);
    for (size_t n = 0; n < N; ++n)
        u_out[n] = g[n] - lambda * d[n];
    free(d); free(w); free(G1); free(G2);
    return 0;
}

/*
 * Duality gap of the ROF step at a dual-feasible p (|p_ij| <= 1), with u = g - lambda div p:
 *   primal  P(u) = 1/2 |u - g|^2 + lambda sum_ij |(grad u)_ij|
 *   dual    D(p) = 1/2 |g|^2 - 1/2 |g - lambda div p|^2
 *   gap     P(u) - D(p) >= 0, and |u - u*|^2 <= 2 gap for the exact minimiser u*.
 * Diagnostic only: it says how far a fixed-iteration step is from the ROF minimiser.
 */
double orc_rof_gap(const double *g, int H, int W, double lambda, const double *p1,
                   const double *p2)
{
    size_t N = (size_t)H * (size_t)W;
    double *d = (double *)malloc(N * sizeof(double));
    double *u = (double *)malloc(N * sizeof(double));
    double *G1 = (double *)malloc(N * sizeof(double));
    double *G2 = (double *)malloc(N * sizeof(double));
    if (!d || !u || !G1 || !G2) {
        free(d); free(u); free(G1); free(G2);
        return NAN;
    }
    orc_div(p1, p2, H, W, d);
    for (size_t n = 0; n < N; ++n)
        u[n] = g[n] - lambda * d[n];
    orc_grad(u, H, W, G1, G2);
    double fid = 0.0, tv = 0.0, gg = 0.0, rr = 0.0;
    for (size_t n = 0; n < N; ++n) {
        fid += 0.5 * (u[n] - g[n]) * (u[n] - g[n]);
        tv += sqrt(G1[n] * G1[n] + G2[n] * G2[n]);
        gg += 0.5 * g[n] * g[n];
        rr += 0.5 * u[n] * u[n]; /* g - lambda div p = u */
    }
    free(d); free(u); free(G1); free(G2);
    return (fid + lambda * tv) - (gg - rr);
}

/* Index m of the band with edges[m] <= t < edges[m+1], or -1 (Eq. spectral_bands, left-closed). */
int orc_band_of(double t, const double *edges, int n_edges)
{
    for (int m = 0; m + 1 < n_edges; ++m)
        if (edges[m] <= t && t < edges[m + 1])
            return m;
    return -1;
}

/*
 * The whole decomposition.
 *   f        H*W input image (row-major)
 *   dt       time step; the ROF weight of every step is lambda = dt
 *   K        number of ROF steps (u_0 = f, ..., u_K); K >= 2
 *   n_inner  Chambolle iterations per step
 *   tau      Chambolle step (0 < tau <= 1/8)
 *   warm_start  1: p carried across steps; 0: p = 0 at the start of every step
 *   edges    n_edges band edges in t (strictly increasing; the last may be +inf)
 * Outputs (all caller-owned):
 *   bands    (n_edges-1)*H*W: b^m = sum_{k: e_m <= t_k < e_{m+1}} phi_k dt
 *   residual H*W: f_r = u_{K-1} - t_{K-1} (u_K - u_{K-1}) / dt
 *   S        K-1 values, S[k-1] = sum_ij |phi_k(i,j)|
 *   u_trace  (K+1)*H*W copies of u_0..u_K, or NULL
 *   filters  n_filters filters: filter_H[q*(K-1) + k-1] = H_q(t_k), filter_res[q] = h_r of
 *            filter q; filtered (n_filters*H*W) receives
 *            f_Hq = sum_{k=1}^{K-1} H_q(t_k) phi_k dt + h_r f_r  (Riemann sum, as the bands)
 *   S_par    K-1 values of the Parseval-type spectrum S_par[k-1] = <phi_k, f> = sum_ij
 *            phi_k(i,j) f(i,j), or NULL. The paper only names this alternative (Burger et al.
 *            2016, cited in Sec. 2.1); read here as the pairing of phi with f, for which
 *            sum_k <phi_k, f> dt + <f_r, f> = |f|^2 follows from the reconstruction.
 * Returns 0, -1 on allocation failure, -2 on invalid arguments.
 */
int orc_decompose_full(const double *f, int H, int W, double dt, int K, int n_inner,
                       double tau, int warm_start, const double *edges, int n_edges,
                       double *bands, double *residual, double *S, double *u_trace,
                       int n_filters, const double *filter_H, const double *filter_res,
                       double *filtered, double *S_par)
{
    if (H < 1 || W < 1 || K < 2 || n_inner < 0 || !(dt > 0.0) || n_edges < 2)
        return -2;
    size_t N = (size_t)H * (size_t)W;
    int n_bands = n_edges - 1;
    double *u_prev = (double *)calloc(N, sizeof(double));
    double *u_cur = (double *)calloc(N, sizeof(double));
    double *u_next = (double *)calloc(N, sizeof(double));
    double *p1 = (double *)calloc(N, sizeof(double));
    double *p2 = (double *)calloc(N, sizeof(double));
    if (!u_prev || !u_cur || !u_next || !p1 || !p2) {
        free(u_prev); free(u_cur); free(u_next); free(p1); free(p2);
        return -1;
    }
    memcpy(u_cur, f, N * sizeof(double)); /* u_0 = f  (Eq. TVflow, u(0) = f) */
    memset(bands, 0, (size_t)n_bands * N * sizeof(double));
    if (n_filters > 0)
        memset(filtered, 0, (size_t)n_filters * N * sizeof(double));
    if (u_trace)
        memcpy(u_trace, u_cur, N * sizeof(double));

    int rc = 0;
    for (int k = 0; k < K; ++k) {
        if (!warm_start) {
            memset(p1, 0, N * sizeof(double));
            memset(p2, 0, N * sizeof(double));
        }
        /* u_{k+1} = argmin_v 1/2 |u_k - v|^2 + dt J_TV(v)   (Eq. ROF) */
        if (orc_chambolle(u_cur, H, W, dt, tau, n_inner, p1, p2, u_next) != 0) {
            rc = -1;
            break;
        }
        if (u_trace)
            memcpy(u_trace + (size_t)(k + 1) * N, u_next, N * sizeof(double));
        if (k >= 1) {
            /* phi_k = t_k u_tt(t_k) by the central second difference (Eq. TVtrafo) */
            double t_k = (double)k * dt;
            int m = orc_band_of(t_k, edges, n_edges);
            double s = 0.0, sp = 0.0;
            for (size_t n = 0; n < N; ++n) {
                double phi = t_k * (u_next[n] - 2.0 * u_cur[n] + u_prev[n]) / (dt * dt);
                s += fabs(phi);                              /* S(t) = |phi(t)|_L1 */
                sp += phi * f[n];                            /* <phi(t), f> */
                if (m >= 0)
                    bands[(size_t)m * N + n] += phi * dt;    /* Eq. spectral_bands */
                for (int q = 0; q < n_filters; ++q)          /* Eq. filteredTVtrafo */
                    filtered[(size_t)q * N + n] +=
                        filter_H[(size_t)q * (K - 1) + (k - 1)] * phi * dt;
            }
            S[k - 1] = s;
            if (S_par)
                S_par[k - 1] = sp;
        }
        double *tmp = u_prev;
        u_prev = u_cur;
        u_cur = u_next;
        u_next = tmp;
    }
    if (rc == 0) {
        /* now u_prev = u_{K-1}, u_cur = u_K; f_r = u(T) - T u_t(T) at T = t_{K-1}
           (Eq. finite_inverse_trafo) */
        double T = (double)(K - 1) * dt;
        for (size_t n = 0; n < N; ++n)
            residual[n] = u_prev[n] - T * (u_cur[n] - u_prev[n]) / dt;
        for (int q = 0; q < n_filters; ++q)
            for (size_t n = 0; n < N; ++n)
                filtered[(size_t)q * N + n] += filter_res[q] * residual[n];
    }
    free(u_prev); free(u_cur); free(u_next); free(p1); free(p2);
    return rc;
}

/* The decomposition with filters, without the Parseval-type spectrum. */
int orc_decompose_filtered(const double *f, int H, int W, double dt, int K, int n_inner,
                           double tau, int warm_start, const double *edges, int n_edges,
                           double *bands, double *residual, double *S, double *u_trace,
                           int n_filters, const double *filter_H, const double *filter_res,
                           double *filtered)
{
    return orc_decompose_full(f, H, W, dt, K, n_inner, tau, warm_start, edges, n_edges, bands,
                              residual, S, u_trace, n_filters, filter_H, filter_res, filtered,
                              NULL);
}

/* The decomposition without filters. */
int orc_decompose(const double *f, int H, int W, double dt, int K, int n_inner, double tau,
                  int warm_start, const double *edges, int n_edges, double *bands,
                  double *residual, double *S, double *u_trace)
{
    return orc_decompose_filtered(f, H, W, dt, K, n_inner, tau, warm_start, edges, n_edges,
                                  bands, residual, S, u_trace, 0, NULL, NULL, NULL);
}

/* ---------------------------------------------------------------------------------------------
 * Training-sample preparation (Sec. 4.1): greyscale crops of a fixed size, some of them taken
 * from a window twice as large and downsampled by 2, and the standardisation of the data set
 * to zero mean and unit standard deviation before the ground-truth bands are computed.
 * Readings: downsampling by s averages each s x s block (area average), the sum taken in
 * row-major order within the block; the standard deviation is the population one (divisor N);
 * a zero standard deviation is replaced by 1; each result is rounded to float32, the type the
 * decomposition reads.
 * -------------------------------------------------------------------------------------------*/

/* out (size x size) = the s-fold block average of the (s*size) x (s*size) window of src
 * (sH x sW, row-major) whose top-left pixel is (y, x). Returns -2 if the window leaves src. */
int orc_crop(const double *src, int sH, int sW, int y, int x, int size, int s, double *out)
{
    if (size < 1 || s < 1 || y < 0 || x < 0 || (long)y + (long)s * size > sH ||
        (long)x + (long)s * size > sW)
        return -2;
    for (int i = 0; i < size; ++i) {
        for (int j = 0; j < size; ++j) {
            double sum = 0.0;
            for (int a = 0; a < s; ++a)
                for (int b = 0; b < s; ++b)
                    sum += src[(size_t)(y + s * i + a) * sW + (x + s * j + b)];
            out[(size_t)i * size + j] = (double)(float)(sum / (double)(s * s));
        }
    }
    return 0;
}

/* Mean and population standard deviation of x[0..n), two passes, sequential sums. */
static void orc_mean_std(const double *x, size_t n, double *mean, double *sd)
{
    double s = 0.0;
    for (size_t i = 0; i < n; ++i) s += x[i];
    const double m = s / (double)n;
    double q = 0.0;
    for (size_t i = 0; i < n; ++i) q += (x[i] - m) * (x[i] - m);
    *mean = m;
    *sd = sqrt(q / (double)n);
}

/* Standardise n_img images of npx pixels each (x, contiguous) into out.
 *   mode 0: out = x;
 *   mode 1: one mean / standard deviation over all n_img * npx values (the data set);
 *           mean_std[0..1] receives them;
 *   mode 2: each image by its own; mean_std[2i..2i+1] receives image i's;
 *   mode 3: by the given mean_std[0], mean_std[1].
 * out = (float)((x - mean) / sd), sd == 0 replaced by 1. Returns -2 on a bad mode. */
int orc_standardize(const double *x, int n_img, size_t npx, int mode, double *mean_std, double *out)
{
    if (n_img < 0 || mode < 0 || mode > 3) return -2;
    const size_t total = (size_t)n_img * npx;
    if (mode == 0) {
        for (size_t i = 0; i < total; ++i) out[i] = x[i];
        return 0;
    }
    for (int c = 0; c < n_img; ++c) {
        double m, sd;
        if (mode == 1) {
            if (c == 0) orc_mean_std(x, total, &mean_std[0], &mean_std[1]);
            m = mean_std[0];
            sd = mean_std[1];
        } else if (mode == 2) {
            orc_mean_std(x + (size_t)c * npx, npx, &mean_std[2 * c], &mean_std[2 * c + 1]);
            m = mean_std[2 * c];
            sd = mean_std[2 * c + 1];
        } else {
            m = mean_std[0];
            sd = mean_std[1];
        }
        if (sd == 0.0) sd = 1.0;
        for (size_t i = 0; i < npx; ++i) {
            const size_t k = (size_t)c * npx + i;
            out[k] = (double)(float)((x[k] - m) / sd);
        }
    }
    return 0;
}

/* ---------------------------------------------------------------------------------------------
 * Other inner solvers of the ROF step (Eq. ROF), for comparison with Chambolle's projection:
 * the fast gradient projection on the same dual problem and the primal-dual hybrid gradient
 * method (the family of the GPU toolbox the paper times in Sec. 4.3), and the duality gap of
 * a primal-dual pair, by which their accuracy is compared.
 * -------------------------------------------------------------------------------------------*/

/* p <- p / max(1, |p|) pointwise (projection onto the unit ball of the isotropic norm). */
static void orc_project_unit(double *p1, double *p2, size_t N)
{
#pragma omp parallel for schedule(static) if (N >= OMP_MIN_PIXELS)
    for (long long n = 0; n < (long long)N; ++n) {
        double norm = sqrt(p1[n] * p1[n] + p2[n] * p2[n]);
        if (norm > 1.0) {
            p1[n] = p1[n] / norm;
            p2[n] = p2[n] / norm;
        }
    }
}

/*
 * n_iter iterations of the fast gradient projection (Beck and Teboulle 2009, FGP) on
 * Chambolle's dual of the ROF step:  min over |p| <= 1 of |g - lambda div p|^2.
 * From r = p_prev = p (the given start) and t = 1, one iteration is
 *   p_new = Pi( r + (1/8) grad(div r - g / lambda) )    (gradient step 1/8 = 1/|div|^2)
 *   t_new = (1 + sqrt(1 + 4 t^2)) / 2
 *   r     = p_new + ((t - 1) / t_new) (p_new - p_prev),  p_prev = p_new,  t = t_new
 * and u = g - lambda div p at the end. p1, p2: start on entry, final p on exit.
 */
int orc_fgp(const double *g, int H, int W, double lambda, int n_iter, double *p1, double *p2,
            double *u_out)
{
    size_t N = (size_t)H * (size_t)W;
    double *r1 = (double *)malloc(N * sizeof(double));
    double *r2 = (double *)malloc(N * sizeof(double));
    double *d = (double *)malloc(N * sizeof(double));
    double *w = (double *)malloc(N * sizeof(double));
    double *G1 = (double *)malloc(N * sizeof(double));
    double *G2 = (double *)malloc(N * sizeof(double));
    double *n1 = (double *)malloc(N * sizeof(double));
    double *n2 = (double *)malloc(N * sizeof(double));
    if (!r1 || !r2 || !d || !w || !G1 || !G2 || !n1 || !n2) {
        free(r1); free(r2); free(d); free(w); free(G1); free(G2); free(n1); free(n2);
        return -1;
    }
    memcpy(r1, p1, N * sizeof(double));
    memcpy(r2, p2, N * sizeof(double));
    double t = 1.0;
    for (int it = 0; it < n_iter; ++it) {
        orc_div(r1, r2, H, W, d);
        for (size_t n = 0; n < N; ++n)
            w[n] = d[n] - g[n] / lambda;
        orc_grad(w, H, W, G1, G2);
        for (size_t n = 0; n < N; ++n) {
            n1[n] = r1[n] + G1[n] / 8.0;
            n2[n] = r2[n] + G2[n] / 8.0;
        }
        orc_project_unit(n1, n2, N);
        double t_new = (1.0 + sqrt(1.0 + 4.0 * t * t)) / 2.0;
        double beta = (t - 1.0) / t_new;
        for (size_t n = 0; n < N; ++n) {
            r1[n] = n1[n] + beta * (n1[n] - p1[n]);
            r2[n] = n2[n] + beta * (n2[n] - p2[n]);
            p1[n] = n1[n];
            p2[n] = n2[n];
        }
        t = t_new;
    }
    orc_div(p1, p2, H, W, d);
    for (size_t n = 0; n < N; ++n)
        u_out[n] = g[n] - lambda * d[n];
    free(r1); free(r2); free(d); free(w); free(G1); free(G2); free(n1); free(n2);
    return 0;
}

/*
 * n_iter iterations of the primal-dual hybrid gradient method (Chambolle and Pock 2011; with
 * gamma > 0 their accelerated variant for a uniformly convex data term) on the saddle-point
 * form of the ROF step,  min_u max_{|y| <= lambda} <grad u, y> + 1/2 |u - g|^2,
 * written with the dual variable p = -y / lambda (|p| <= 1, the same p as Chambolle's, so
 * that u(p) = g - lambda div p). From (u, ubar = u, p) and steps (tau, sigma):
 *   p     = Pi( p - (sigma / lambda) grad ubar )
 *   u_new = (u - tau lambda div p + tau g) / (1 + tau)
 *   theta = 1 / sqrt(1 + 2 gamma tau)   (theta = 1 when gamma = 0)
 *   ubar  = u_new + theta (u_new - u),  u = u_new,  tau = theta tau,  sigma = sigma / theta
 * Convergence needs tau sigma |grad|^2 <= 1, |grad|^2 <= 8. u, p1, p2: start on entry, final
 * iterates on exit.
 */
int orc_pdhg(const double *g, int H, int W, double lambda, int n_iter, double tau, double sigma,
             double gamma, double *u, double *p1, double *p2)
{
    size_t N = (size_t)H * (size_t)W;
    double *ub = (double *)malloc(N * sizeof(double));
    double *d = (double *)malloc(N * sizeof(double));
    double *G1 = (double *)malloc(N * sizeof(double));
    double *G2 = (double *)malloc(N * sizeof(double));
    if (!ub || !d || !G1 || !G2) {
        free(ub); free(d); free(G1); free(G2);
        return -1;
    }
    memcpy(ub, u, N * sizeof(double));
    for (int it = 0; it < n_iter; ++it) {
        orc_grad(ub, H, W, G1, G2);
        for (size_t n = 0; n < N; ++n) {
            p1[n] = p1[n] - (sigma / lambda) * G1[n];
            p2[n] = p2[n] - (sigma / lambda) * G2[n];
        }
        orc_project_unit(p1, p2, N);
        orc_div(p1, p2, H, W, d);
        double theta = gamma > 0.0 ? 1.0 / sqrt(1.0 + 2.0 * gamma * tau) : 1.0;
        for (size_t n = 0; n < N; ++n) {
            double un = (u[n] - tau * lambda * d[n] + tau * g[n]) / (1.0 + tau);
            ub[n] = un + theta * (un - u[n]);
            u[n] = un;
        }
        tau = theta * tau;
        sigma = sigma / theta;
    }
    free(ub); free(d); free(G1); free(G2);
    return 0;
}

/*
 * Duality gap of a primal-dual pair (u, p) of the ROF step, |p| <= 1:
 *   P(u) - D(p) = 1/2 |u - g|^2 + lambda sum |grad u|  -  (1/2 |g|^2 - 1/2 |g - lambda div p|^2)
 * >= P(u) - P(u*) >= 1/2 |u - u*|^2.
 */
double orc_rof_gap_pair(const double *g, int H, int W, double lambda, const double *u,
                        const double *p1, const double *p2)
{
    size_t N = (size_t)H * (size_t)W;
    double *d = (double *)malloc(N * sizeof(double));
    double *G1 = (double *)malloc(N * sizeof(double));
    double *G2 = (double *)malloc(N * sizeof(double));
    if (!d || !G1 || !G2) {
        free(d); free(G1); free(G2);
        return NAN;
    }
    orc_div(p1, p2, H, W, d);
    orc_grad(u, H, W, G1, G2);
    double fid = 0.0, tv = 0.0, gg = 0.0, rr = 0.0;
    for (size_t n = 0; n < N; ++n) {
        double r = g[n] - lambda * d[n];
        fid += 0.5 * (u[n] - g[n]) * (u[n] - g[n]);
        tv += sqrt(G1[n] * G1[n] + G2[n] * G2[n]);
        gg += 0.5 * g[n] * g[n];
        rr += 0.5 * r * r;
    }
    free(d); free(G1); free(G2);
    return (fid + lambda * tv) - (gg - rr);
}
