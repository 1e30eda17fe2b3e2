/*
 * rt_oracle.c -- plain, slow FP64 CPU oracle for point-based ray tracing of
 * 3D Gaussians (visibility precompute).  TEST INFRASTRUCTURE ONLY: it is
 * called by tests/, by the CUDA-path smoke check and by the CPU-baseline leg
 * of bench.py, never by the product path.  It shares no code, header or table
 * with the CUDA library.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fno-fast-math -fPIC -shared.
 * -ffp-contract=off matters: the float32 parts below (ray origins, Morton
 * quantisation) are defined as separately rounded IEEE operations.
 *
 * What each function follows
 *   rot_from_quat      Sec. 3.1: Sigma = R S S^T R^T from a unit quaternion q
 *                      (w first) and a scale vector s.
 *   oracle_trace       Eq. 1 (Gaussian), Eq. 13-14 (equivalent intersection at
 *                      the Gaussian's peak along the ray; the covariance in
 *                      Eq. 14 is read as Sigma^-1, which is what makes r_x the
 *                      peak), Eq. 2 / Eq. 15 (T = prod (1 - alpha_j), order
 *                      independent, Sec. 4.1), early termination below T_min
 *                      (Sec. 4.1).  Brute force: every ray against every
 *                      Gaussian, no BVH.
 *   oracle_trace_grad  analytic gradient of L = sum_r g_r T_r with respect to
 *                      opacity, mean, scale, quaternion and ray origin (the
 *                      paper freezes geometry after the precompute, Sec. 4.2;
 *                      the adjoint is the plain chain rule of the forward).
 *   oracle_dir_rays    rays cast from each Gaussian in a fixed direction set
 *                      (Sec. 4.2, Sec. 3.3), origin offset along the direction.
 *   oracle_env_rays    shadow rays importance-sampled from an environment map
 *                      (the direct light of Eq. 8), Philox4x64-10 counter-based
 *                      random numbers (Salmon et al. 2011).
 *   oracle_morton / oracle_lbvh
 *                      the binary radix tree of Sec. 4.1 (Karras 2012): 30-bit
 *                      Morton codes of the centroids, keys code<<32|index,
 *                      sorted, internal nodes by the longest-common-prefix
 *                      split rule; exact FP64 leaf boxes (K-sigma extents).
 *   oracle_bvh_*       the same visibility as oracle_trace, found through the
 *                      LBVH twin (Sec. 4.1: rays traced through a BVH over the
 *                      Gaussians' boxes) with boxes that cover every candidate
 *                      brute force accepts or flags; pinned against
 *                      oracle_trace, it reaches every ray of the large scenes.
 *   oracle_hemi_rays / oracle_pbr
 *                      the hemisphere direction set about each Gaussian's
 *                      normal (Sec. 3.3, Fibonacci sampling) and the
 *                      per-Gaussian PBR colour of Eq. 10 (simplified Disney
 *                      BRDF of Eq. 9, light of Eq. 8: visibility x a global
 *                      environment map plus degree-2 SH indirect light).
 *   oracle_mlp_*       the visibility surrogate (not in the paper): frequency
 *                      encoding, 4x128 ReLU MLP, sigmoid, BCE, Adam; bf16
 *                      rounding emulated where the GPU stores bf16, FP64
 *                      accumulation.
 *
 * Readings where the paper is silent:
 *   - accept Gaussian j on a ray iff t* > 0, m^2 <= k_sigma^2 and
 *     alpha >= alpha_min (alpha = o * exp(-m^2/2)); no clamp of alpha;
 *   - the ray's own source Gaussian is excluded by index;
 *   - early termination snaps T to 0 when the exact product is < T_min
 *     (T_min = 0 disables it); with a monotone product this is order-free;
 *   - rays with a candidate inside a rounding band around a threshold are
 *     flagged (bits of flags[]), so tests can exclude and count them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Gaussian geometry in FP64                                                 */
/* ------------------------------------------------------------------------ */

/* Rotation matrix of the normalised quaternion (w, x, y, z); R[3*i+j] is
 * row i, column j.  The columns are the Gaussian's local axes in world space. */
static void rot_from_quat(const double qin[4], double R[9], double qhat[4], double *qnorm)
{
    double n = sqrt(qin[0] * qin[0] + qin[1] * qin[1] + qin[2] * qin[2] + qin[3] * qin[3]);
    double w = qin[0] / n, x = qin[1] / n, y = qin[2] / n, z = qin[3] / n;
    R[0] = 1.0 - 2.0 * (y * y + z * z); R[1] = 2.0 * (x * y - w * z);       R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);       R[4] = 1.0 - 2.0 * (x * x + z * z); R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);       R[7] = 2.0 * (y * z + w * x);       R[8] = 1.0 - 2.0 * (x * x + y * y);
    if (qhat) { qhat[0] = w; qhat[1] = x; qhat[2] = y; qhat[3] = z; }
    if (qnorm) *qnorm = n;
}

/* Exported for tests: R of a quaternion, FP64. */
void oracle_rotation(const double *q, double *R) { rot_from_quat(q, R, NULL, NULL); }

typedef struct {
    double mu[3], R[9], s[3], o;
} gauss64;

static gauss64 *load_gaussians(int64_t n, const double *mean, const double *scale,
                               const double *quat, const double *opac)
{
    gauss64 *g = (gauss64 *)malloc((size_t)(n > 0 ? n : 1) * sizeof(gauss64));
    for (int64_t j = 0; j < n; ++j) {
        double q[4] = {quat[4 * j], quat[4 * j + 1], quat[4 * j + 2], quat[4 * j + 3]};
        rot_from_quat(q, g[j].R, NULL, NULL);
        for (int k = 0; k < 3; ++k) {
            g[j].mu[k] = mean[3 * j + k];
            g[j].s[k] = scale[3 * j + k];
        }
        g[j].o = opac[j];
    }
    return g;
}

/* Peak response of Gaussian g along the ray (ro, rd) -- Eq. 13-14 with
 * Sigma^-1.  In the Gaussian's whitened frame u(x) = S^-1 R^T (x - mu) the
 * Mahalanobis distance is |u|^2, so along x = ro + t rd it is the quadratic
 * |u_o + t u_d|^2 whose minimiser is t* = -(u_o . u_d) / (u_d . u_d).
 * Returns m^2 at t*, writes t*, and (optionally) e = x(t*) - mu. */
static double peak_m2(const gauss64 *g, const double ro[3], const double rd[3],
                      double *t_out, double e_out[3])
{
    double dl[3] = {ro[0] - g->mu[0], ro[1] - g->mu[1], ro[2] - g->mu[2]};
    double uo[3], ud[3];
    for (int k = 0; k < 3; ++k) {
        /* column k of R is local axis k: (R^T v)_k = sum_i R[i][k] v_i */
        double a = g->R[0 * 3 + k] * dl[0] + g->R[1 * 3 + k] * dl[1] + g->R[2 * 3 + k] * dl[2];
        double b = g->R[0 * 3 + k] * rd[0] + g->R[1 * 3 + k] * rd[1] + g->R[2 * 3 + k] * rd[2];
        uo[k] = a / g->s[k];
        ud[k] = b / g->s[k];
    }
    double aa = ud[0] * ud[0] + ud[1] * ud[1] + ud[2] * ud[2];
    double bb = uo[0] * ud[0] + uo[1] * ud[1] + uo[2] * ud[2];
    double t = -bb / aa;
    double m2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        double u = uo[k] + t * ud[k];
        m2 += u * u;
    }
    if (t_out) *t_out = t;
    if (e_out)
        for (int k = 0; k < 3; ++k) e_out[k] = dl[k] + t * rd[k];
    return m2;
}

/* Band flags (bit meanings) */
#define ORC_FLAG_M2 1u     /* a candidate has |m^2 - K^2| <= band_m2          */
#define ORC_FLAG_ALPHA 2u  /* a candidate has |alpha - alpha_min| <= band_a    */
#define ORC_FLAG_T 4u      /* a candidate has |t*| <= band_t                   */
#define ORC_FLAG_TMIN 8u   /* |T_exact - T_min| <= band_T                      */

/*
 * Brute-force visibility.  For each ray r (origin ray_o[r], direction ray_d[r],
 * source Gaussian ray_src[r] or -1; FP64 inputs, normally float32 widened):
 *   T_exact[r] = prod over accepted j (ascending j) of (1 - alpha_j)
 *   T[r]       = 0 if T_exact < t_min else T_exact
 *   hits[r]    = number of accepted Gaussians
 *   flags[r]   = band bits above (band widths are arguments).
 *   T_lo[r], T_hi[r] = the products with every candidate that set a band bit
 *                (a "borderline" candidate: one threshold test within its
 *                band, the others passed within theirs) taken / left out,
 *                and every other candidate as in T_exact: an exact float32
 *                evaluation may take any subset of the borderline ones, so
 *                its unsnapped product lies in [T_lo, T_hi] (equal to
 *                T_exact when flags has no candidate bit).
 *   n_border[r] = the number of those borderline candidates: such an
 *                evaluation accepts hits[r] of them give or take n_border[r].
 * Output pointers other than T may be NULL.
 */
void oracle_trace(int64_t n, const double *mean, const double *scale, const double *quat,
                  const double *opac, int64_t n_rays, const double *ray_o, const double *ray_d,
                  const int32_t *ray_src, double k_sigma, double alpha_min, double t_min,
                  double band_m2, double band_alpha, double band_t, double band_T,
                  double *T, double *T_exact, int32_t *hits, uint32_t *flags, double *T_lo, double *T_hi,
                  int32_t *n_border)
{
    gauss64 *g = load_gaussians(n, mean, scale, quat, opac);
    const double K2 = k_sigma * k_sigma;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < n_rays; ++r) {
        double ro[3] = {ray_o[3 * r], ray_o[3 * r + 1], ray_o[3 * r + 2]};
        double rd[3] = {ray_d[3 * r], ray_d[3 * r + 1], ray_d[3 * r + 2]};
        int64_t src = ray_src ? ray_src[r] : -1;
        double tr = 1.0, tlo = 1.0, thi = 1.0;
        int32_t nh = 0, nb = 0;
        uint32_t fl = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == src) continue;
            double t;
            double m2 = peak_m2(&g[j], ro, rd, &t, NULL);
            double alpha = g[j].o * exp(-0.5 * m2);
            int ok_t = t > 0.0, ok_m = m2 <= K2, ok_a = alpha >= alpha_min;
            /* near-threshold candidates: the other two tests pass within their bands */
            int near_t = fabs(t) <= band_t, near_m = fabs(m2 - K2) <= band_m2,
                near_a = fabs(alpha - alpha_min) <= band_alpha;
            int lo_t = ok_t || near_t, lo_m = ok_m || near_m, lo_a = ok_a || near_a;
            int border = 0;
            if (near_t && lo_m && lo_a) { fl |= ORC_FLAG_T; border = 1; }
            if (near_m && lo_t && lo_a) { fl |= ORC_FLAG_M2; border = 1; }
            if (near_a && lo_t && lo_m) { fl |= ORC_FLAG_ALPHA; border = 1; }
            if (ok_t && ok_m && ok_a) {
                tr *= (1.0 - alpha);
                ++nh;
            }
            if (border) {
                tlo *= (1.0 - alpha);
                ++nb;
            } else if (ok_t && ok_m && ok_a) {
                tlo *= (1.0 - alpha);
                thi *= (1.0 - alpha);
            }
        }
        if (t_min > 0.0 && fabs(tr - t_min) <= band_T) fl |= ORC_FLAG_TMIN;
        if (T_lo) T_lo[r] = tlo;
        if (T_hi) T_hi[r] = thi;
        if (T_exact) T_exact[r] = tr;
        T[r] = (tr < t_min) ? 0.0 : tr;
        if (hits) hits[r] = nh;
        if (flags) flags[r] = fl;
        if (n_border) n_border[r] = nb;
    }
    free(g);
}

/*
 * List the accepted Gaussians of each ray (ascending index): for ray r,
 * ids[r*cap .. r*cap + min(count[r], cap)) and count[r] = total accepted.
 * Same acceptance rule as oracle_trace, no early termination.
 */
void oracle_trace_hits(int64_t n, const double *mean, const double *scale, const double *quat,
                       const double *opac, int64_t n_rays, const double *ray_o, const double *ray_d,
                       const int32_t *ray_src, double k_sigma, double alpha_min,
                       int32_t cap, int32_t *ids, int32_t *count)
{
    gauss64 *g = load_gaussians(n, mean, scale, quat, opac);
    const double K2 = k_sigma * k_sigma;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < n_rays; ++r) {
        double ro[3] = {ray_o[3 * r], ray_o[3 * r + 1], ray_o[3 * r + 2]};
        double rd[3] = {ray_d[3 * r], ray_d[3 * r + 1], ray_d[3 * r + 2]};
        int64_t src = ray_src ? ray_src[r] : -1;
        int32_t c = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == src) continue;
            double t;
            double m2 = peak_m2(&g[j], ro, rd, &t, NULL);
            double alpha = g[j].o * exp(-0.5 * m2);
            if (t > 0.0 && m2 <= K2 && alpha >= alpha_min) {
                if (c < cap) ids[r * (int64_t)cap + c] = (int32_t)j;
                ++c;
            }
        }
        count[r] = c;
    }
    free(g);
}

/* Chain rule through R(q_hat) and q_hat = q / |q|: given G = dL/dR (row-major
 * 3x3), accumulate dL/dq for the un-normalised q. */
static void quat_backward(const double qhat[4], double qnorm, const double G[9], double dq[4])
{
    double w = qhat[0], x = qhat[1], y = qhat[2], z = qhat[3];
    double gw = 2.0 * (-z * G[1] + y * G[2] + z * G[3] - x * G[5] - y * G[6] + x * G[7]);
    double gx = 2.0 * (y * G[1] + z * G[2] + y * G[3] - 2.0 * x * G[4] - w * G[5] + z * G[6] + w * G[7] - 2.0 * x * G[8]);
    double gy = 2.0 * (-2.0 * y * G[0] + x * G[1] + w * G[2] + x * G[3] + z * G[5] - w * G[6] + z * G[7] - 2.0 * y * G[8]);
    double gz = 2.0 * (-2.0 * z * G[0] - w * G[1] + x * G[2] + w * G[3] - 2.0 * z * G[4] + y * G[5] + x * G[6] + y * G[7]);
    double dot = w * gw + x * gx + y * gy + z * gz;
    dq[0] += (gw - w * dot) / qnorm;
    dq[1] += (gx - x * dot) / qnorm;
    dq[2] += (gy - y * dot) / qnorm;
    dq[3] += (gz - z * dot) / qnorm;
}

/*
 * Analytic gradient of L = sum_r dL_dT[r] * T[r] (T as in oracle_trace; a ray
 * whose T was snapped to 0 by early termination contributes nothing).
 * With P_j = prod_{i != j} (1 - alpha_i):  dT/dalpha_j = -P_j,
 *   alpha = o exp(-m^2/2):  dalpha/do = exp(-m^2/2),  dalpha/dm^2 = -alpha/2.
 * m^2 is stationary in t at t*, so with x = ro + t* rd held fixed and
 * e = x - mu, u = S^-1 R^T e:
 *   dm^2/dmu  = -2 Sigma^-1 e,   dm^2/dro = +2 Sigma^-1 e,
 *   dm^2/ds_k = -2 u_k^2 / s_k,  dm^2/dR_ik = 2 e_i u_k / s_k.
 * Outputs (FP64, zeroed here): d_mean[n,3], d_scale[n,3], d_quat[n,4],
 * d_opac[n], d_ray_o[n_rays,3] (may be NULL).
 */
void oracle_trace_grad(int64_t n, const double *mean, const double *scale, const double *quat,
                       const double *opac, int64_t n_rays, const double *ray_o, const double *ray_d,
                       const int32_t *ray_src, double k_sigma, double alpha_min, double t_min,
                       const double *dL_dT, double *d_mean, double *d_scale, double *d_quat,
                       double *d_opac, double *d_ray_o)
{
    gauss64 *g = load_gaussians(n, mean, scale, quat, opac);
    double *qhat = (double *)malloc((size_t)(n > 0 ? n : 1) * 5 * sizeof(double));
    for (int64_t j = 0; j < n; ++j) {
        double q[4] = {quat[4 * j], quat[4 * j + 1], quat[4 * j + 2], quat[4 * j + 3]};
        double Rt[9];
        rot_from_quat(q, Rt, &qhat[5 * j], &qhat[5 * j + 4]);
    }
    const double K2 = k_sigma * k_sigma;
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    const int64_t per = n * 11;
    double *acc = (double *)calloc((size_t)nthreads * (size_t)(per > 0 ? per : 1), sizeof(double));
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *A = acc + (size_t)tid * (size_t)per;
        int32_t cap = 64;
        int32_t *list = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
        double *alist = (double *)malloc(sizeof(double) * (size_t)cap);
#pragma omp for schedule(dynamic, 32)
        for (int64_t r = 0; r < n_rays; ++r) {
            double ro[3] = {ray_o[3 * r], ray_o[3 * r + 1], ray_o[3 * r + 2]};
            double rd[3] = {ray_d[3 * r], ray_d[3 * r + 1], ray_d[3 * r + 2]};
            int64_t src = ray_src ? ray_src[r] : -1;
            double tr = 1.0;
            int32_t c = 0;
            for (int64_t j = 0; j < n; ++j) {
                if (j == src) continue;
                double t;
                double m2 = peak_m2(&g[j], ro, rd, &t, NULL);
                double alpha = g[j].o * exp(-0.5 * m2);
                if (t > 0.0 && m2 <= K2 && alpha >= alpha_min) {
                    if (c == cap) {
                        cap *= 2;
                        list = (int32_t *)realloc(list, sizeof(int32_t) * (size_t)cap);
                        alist = (double *)realloc(alist, sizeof(double) * (size_t)cap);
                    }
                    list[c] = (int32_t)j;
                    alist[c] = alpha;
                    ++c;
                    tr *= (1.0 - alpha);
                }
            }
            if (d_ray_o) d_ray_o[3 * r] = d_ray_o[3 * r + 1] = d_ray_o[3 * r + 2] = 0.0;
            if (tr < t_min) continue; /* snapped: locally constant T = 0 */
            for (int32_t h = 0; h < c; ++h) {
                int64_t j = list[h];
                /* product of the other factors, formed directly (no division) */
                double P = 1.0;
                for (int32_t h2 = 0; h2 < c; ++h2)
                    if (h2 != h) P *= (1.0 - alist[h2]);
                double gA = dL_dT[r] * (-P); /* dL/dalpha_j */
                double t, e[3];
                double m2 = peak_m2(&g[j], ro, rd, &t, e);
                double ex = exp(-0.5 * m2);
                double alpha = g[j].o * ex;
                double gM = gA * (-0.5 * alpha); /* dL/dm^2 */
                const double *R = g[j].R;
                double u[3], w[3];
                for (int k = 0; k < 3; ++k) {
                    u[k] = (R[0 * 3 + k] * e[0] + R[1 * 3 + k] * e[1] + R[2 * 3 + k] * e[2]) / g[j].s[k];
                    w[k] = u[k] / g[j].s[k]; /* (S^-2 R^T e)_k */
                }
                double sie[3]; /* Sigma^-1 e = R S^-2 R^T e */
                for (int i = 0; i < 3; ++i) sie[i] = R[i * 3 + 0] * w[0] + R[i * 3 + 1] * w[1] + R[i * 3 + 2] * w[2];
                double *Am = A + j * 11; /* layout: mean 3, scale 3, quat 4, opac 1 */
                for (int i = 0; i < 3; ++i) Am[i] += gM * (-2.0 * sie[i]);
                for (int k = 0; k < 3; ++k) Am[3 + k] += gM * (-2.0 * u[k] * u[k] / g[j].s[k]);
                double G[9];
                for (int i = 0; i < 3; ++i)
                    for (int k = 0; k < 3; ++k) G[i * 3 + k] = gM * 2.0 * e[i] * w[k];
                double dq[4] = {0, 0, 0, 0};
                quat_backward(&qhat[5 * j], qhat[5 * j + 4], G, dq);
                for (int k = 0; k < 4; ++k) Am[6 + k] += dq[k];
                Am[10] += gA * ex;
                if (d_ray_o)
                    for (int i = 0; i < 3; ++i) d_ray_o[3 * r + i] += gM * (2.0 * sie[i]);
            }
        }
        free(list);
        free(alist);
    }
    for (int64_t j = 0; j < n; ++j) {
        double s[11] = {0};
        for (int th = 0; th < nthreads; ++th)
            for (int k = 0; k < 11; ++k) s[k] += acc[(size_t)th * (size_t)per + (size_t)j * 11 + (size_t)k];
        for (int k = 0; k < 3; ++k) d_mean[3 * j + k] = s[k];
        for (int k = 0; k < 3; ++k) d_scale[3 * j + k] = s[3 + k];
        for (int k = 0; k < 4; ++k) d_quat[4 * j + k] = s[6 + k];
        d_opac[j] = s[10];
    }
    free(acc);
    free(qhat);
    free(g);
}

/* ------------------------------------------------------------------------ */
/* Ray sets                                                                  */
/* ------------------------------------------------------------------------ */

/*
 * Rays cast from each Gaussian in a fixed direction set (Sec. 4.2).  Ray id
 * r = g*K + k: source Gaussian g, direction dirs[k].  The origin is the mean
 * pushed along the direction by eps, in float32 with two roundings:
 * o = fl(mu + fl(eps * d)).  Only the listed ids are produced.
 */
void oracle_dir_rays(int64_t n, const float *mean, int32_t K, const float *dirs, float eps,
                     const int64_t *ids, int64_t m, float *ray_o, float *ray_d, int32_t *ray_src)
{
    (void)n;
    for (int64_t i = 0; i < m; ++i) {
        int64_t r = ids[i];
        int64_t gi = r / K;
        int32_t k = (int32_t)(r % K);
        for (int c = 0; c < 3; ++c) {
            float d = dirs[3 * k + c];
            float off = eps * d;
            float o = mean[3 * gi + c] + off;
            ray_o[3 * i + c] = o;
            ray_d[3 * i + c] = d;
        }
        ray_src[i] = (int32_t)gi;
    }
}

/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11): counter c[4], key k[2], ten rounds of two 64x64->128
 * multiplies, key bumped by the Weyl constants between rounds. */
static void philox4x64_10(const uint64_t cin[4], const uint64_t kin[2], uint64_t out[4])
{
    uint64_t c0 = cin[0], c1 = cin[1], c2 = cin[2], c3 = cin[3];
    uint64_t k0 = kin[0], k1 = kin[1];
    for (int round = 0; round < 10; ++round) {
        unsigned __int128 p0 = (unsigned __int128)0xD2E7470EE14C6C93ull * c0;
        unsigned __int128 p1 = (unsigned __int128)0xCA5A826395121157ull * c2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B97F4A7C15ull;
        k1 += 0xBB67AE8584CAA73Bull;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void oracle_philox(const uint64_t *ctr, const uint64_t *key, uint64_t *out) { philox4x64_10(ctr, key, out); }

/*
 * Shadow rays toward directions importance-sampled from an environment map.
 * Pixel (i, j) of the h x w map is drawn with probability proportional to
 * radiance[i][j] * solid_angle[i][j]: the cumulative sums are formed in FP64,
 * row-major, in index order, and divided by the total; the pixel is the first
 * with cdf > u0.  Inside the pixel the direction is the normalised bilinear
 * blend of its four corner directions, in float32 with separately rounded
 * operations:
 *   top = c00 + a*(c01 - c00), bot = c10 + a*(c11 - c10), v = top + b*(bot - top),
 *   d = v / sqrt((vx*vx + vy*vy) + vz*vz).
 * Random numbers: Philox4x64-10 with counter (r, 0, 0, 0) and key (seed, 0)
 * for ray id r = g*S + s, outputs x0..x3:
 *   u0 = (x0 >> 11) * 2^-53 (FP64),
 *   a = (x1 >> 40) * 2^-24, b = (x2 >> 40) * 2^-24 (float32, exact).
 * Origin as in oracle_dir_rays.
 */
void oracle_env_rays(int64_t n, const float *mean, int32_t h, int32_t w, const double *radiance,
                     const double *solid_angle, const float *corners, uint32_t seed, int32_t S,
                     float eps, const int64_t *ids, int64_t m, float *ray_o, float *ray_d,
                     int32_t *ray_src)
{
    (void)n;
    int64_t np = (int64_t)h * w;
    double *cdf = (double *)malloc(sizeof(double) * (size_t)np);
    double run = 0.0;
    for (int64_t p = 0; p < np; ++p) {
        run += radiance[p] * solid_angle[p];
        cdf[p] = run;
    }
    for (int64_t p = 0; p < np; ++p) cdf[p] = cdf[p] / run;
    for (int64_t i = 0; i < m; ++i) {
        int64_t r = ids[i];
        int64_t gi = r / S;
        uint64_t ctr[4] = {(uint64_t)r, 0u, 0u, 0u};
        uint64_t key[2] = {(uint64_t)seed, 0u};
        uint64_t x[4];
        philox4x64_10(ctr, key, x);
        double u0 = (double)(x[0] >> 11) * (1.0 / 9007199254740992.0);
        /* first pixel with cdf > u0, by a plain linear scan */
        int64_t p = 0;
        while (p < np - 1 && !(cdf[p] > u0)) ++p;
        int64_t pi = p / w, pj = p % w;
        float a = (float)(x[1] >> 40) * (1.0f / 16777216.0f);
        float b = (float)(x[2] >> 40) * (1.0f / 16777216.0f);
        const float *c00 = corners + 3 * ((pi * (w + 1)) + pj);
        const float *c01 = corners + 3 * ((pi * (w + 1)) + pj + 1);
        const float *c10 = corners + 3 * (((pi + 1) * (w + 1)) + pj);
        const float *c11 = corners + 3 * (((pi + 1) * (w + 1)) + pj + 1);
        float v[3];
        for (int c = 0; c < 3; ++c) {
            float d0 = c01[c] - c00[c];
            float t0 = a * d0;
            float top = c00[c] + t0;
            float d1 = c11[c] - c10[c];
            float t1 = a * d1;
            float bot = c10[c] + t1;
            float d2 = bot - top;
            float t2 = b * d2;
            v[c] = top + t2;
        }
        float xx = v[0] * v[0];
        float yy = v[1] * v[1];
        float zz = v[2] * v[2];
        float ss = xx + yy;
        ss = ss + zz;
        float len = sqrtf(ss);
        for (int c = 0; c < 3; ++c) {
            float d = v[c] / len;
            float off = eps * d;
            ray_d[3 * i + c] = d;
            ray_o[3 * i + c] = mean[3 * gi + c] + off;
        }
        ray_src[i] = (int32_t)gi;
    }
    free(cdf);
}

/* ------------------------------------------------------------------------ */
/* LBVH twin (Sec. 4.1, binary radix tree of Karras 2012)                    */
/* ------------------------------------------------------------------------ */

static uint32_t spread10(uint32_t v)
{
    /* bit b of v goes to bit 3b */
    uint32_t r = 0;
    for (int b = 0; b < 10; ++b) r |= ((v >> b) & 1u) << (3 * b);
    return r;
}

/*
 * 30-bit Morton codes of the centroids (= means).  Scene bounds lo/hi are the
 * per-axis min/max of the means; per axis, in float32 with IEEE rounding:
 * ext = hi - lo; u = (mu - lo) / ext; v = u * 1024; q = clamp(floor(v), 0, 1023)
 * (q = 0 when ext == 0).  code = x bits at 3b+2, y at 3b+1, z at 3b.
 */
void oracle_morton(int64_t n, const float *mean, uint32_t *codes, float *lo_out, float *hi_out)
{
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < 3; ++c) {
            float v = mean[3 * i + c];
            if (v < lo[c]) lo[c] = v;
            if (v > hi[c]) hi[c] = v;
        }
    for (int64_t i = 0; i < n; ++i) {
        uint32_t q[3];
        for (int c = 0; c < 3; ++c) {
            float ext = hi[c] - lo[c];
            if (ext == 0.0f) { q[c] = 0; continue; }
            float num = mean[3 * i + c] - lo[c];
            float u = num / ext;
            float v = u * 1024.0f;
            float f = floorf(v);
            int32_t qi = (int32_t)f;
            if (qi < 0) qi = 0;
            if (qi > 1023) qi = 1023;
            q[c] = (uint32_t)qi;
        }
        codes[i] = (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
    }
    if (lo_out) for (int c = 0; c < 3; ++c) lo_out[c] = lo[c];
    if (hi_out) for (int c = 0; c < 3; ++c) hi_out[c] = hi[c];
}

static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

static int clz64(uint64_t x)
{
    int c = 0;
    for (int b = 63; b >= 0; --b) {
        if ((x >> b) & 1u) break;
        ++c;
    }
    return c;
}

static int delta(const uint64_t *k, int64_t n, int64_t i, int64_t j)
{
    if (j < 0 || j >= n) return -1;
    return clz64(k[i] ^ k[j]);
}

#define ORC_LEAF 0x80000000u

/*
 * Binary radix tree over the unique keys code<<32 | index, sorted ascending.
 * Internal node i (0..n-2) covers a key range with i at one end; its split is
 * the last position sharing the range's longest common prefix.  Children:
 * left = split (a leaf iff the range starts there), right = split+1 (a leaf
 * iff the range ends there).  Leaf refs carry bit 31.  parent[] has n-1
 * internal entries followed by n leaf entries (root's parent = -1).
 */
void oracle_lbvh(int64_t n, const float *mean, uint64_t *keys, int32_t *left, int32_t *right,
                 int32_t *parent)
{
    uint32_t *codes = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    oracle_morton(n, mean, codes, NULL, NULL);
    for (int64_t i = 0; i < n; ++i) keys[i] = ((uint64_t)codes[i] << 32) | (uint64_t)i;
    qsort(keys, (size_t)n, sizeof(uint64_t), cmp_u64);
    free(codes);
    if (n <= 0) return;
    parent[n - 1] = -1; /* n == 1: the single leaf is the root */
    if (n == 1) return;
    parent[0] = -1;
    for (int64_t i = 0; i < n - 1; ++i) {
        int d = (delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1)) >= 0 ? 1 : -1;
        int dmin = delta(keys, n, i, i - d);
        int64_t lmax = 2;
        while (delta(keys, n, i, i + lmax * d) > dmin) lmax *= 2;
        int64_t l = 0;
        for (int64_t t = lmax / 2; t >= 1; t /= 2)
            if (delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
        int64_t j = i + l * d;
        int dnode = delta(keys, n, i, j);
        int64_t s = 0, t = l;
        for (;;) {
            t = (t + 1) / 2;
            if (delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
            if (t == 1) break;
        }
        int64_t gamma = i + s * d + (d < 0 ? -1 : 0);
        int64_t first = i < j ? i : j, last = i < j ? j : i;
        if (first == gamma) {
            left[i] = (int32_t)(ORC_LEAF | (uint32_t)gamma);
            parent[(n - 1) + gamma] = (int32_t)i;
        } else {
            left[i] = (int32_t)gamma;
            parent[gamma] = (int32_t)i;
        }
        if (last == gamma + 1) {
            right[i] = (int32_t)(ORC_LEAF | (uint32_t)(gamma + 1));
            parent[(n - 1) + gamma + 1] = (int32_t)i;
        } else {
            right[i] = (int32_t)(gamma + 1);
            parent[gamma + 1] = (int32_t)i;
        }
    }
}

/*
 * Exact FP64 axis-aligned box of each Gaussian's support {m^2 <= K_j^2}:
 * half-extent along world axis i is K_j * sqrt(Sigma_ii), Sigma_ii =
 * sum_k R_ik^2 s_k^2.  K_j = k_sigma (box_mode 0) or, with box_mode 1,
 * min(k_sigma, sqrt(2 ln(o_j / alpha_min))) and an empty box (lo > hi) when
 * o_j < alpha_min: beyond that radius alpha < alpha_min, so the accepted set
 * is unchanged.  box[j] = (lo_x, lo_y, lo_z, hi_x, hi_y, hi_z).
 */
void oracle_leaf_boxes(int64_t n, const double *mean, const double *scale, const double *quat,
                       const double *opac, double k_sigma, double alpha_min, int32_t box_mode,
                       double *box)
{
    for (int64_t j = 0; j < n; ++j) {
        double q[4] = {quat[4 * j], quat[4 * j + 1], quat[4 * j + 2], quat[4 * j + 3]}, R[9];
        rot_from_quat(q, R, NULL, NULL);
        double K = k_sigma;
        int empty = 0;
        if (box_mode == 1) {
            double o = opac[j];
            if (o < alpha_min) empty = 1;
            else {
                double kk = 2.0 * log(o / alpha_min);
                if (kk < K * K) K = sqrt(kk);
            }
        }
        for (int i = 0; i < 3; ++i) {
            double sii = 0.0;
            for (int k = 0; k < 3; ++k) {
                double v = R[i * 3 + k] * scale[3 * j + k];
                sii += v * v;
            }
            double h = K * sqrt(sii);
            box[6 * j + i] = empty ? INFINITY : mean[3 * j + i] - h;
            box[6 * j + 3 + i] = empty ? -INFINITY : mean[3 * j + i] + h;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* CPU BVH tracer: oracle_trace's visibility through the LBVH twin           */
/* ------------------------------------------------------------------------ */

/*
 * Sec. 4.1 finds the Gaussians a ray meets by tracing it through a BVH over
 * their bounding boxes; the visibility is still the product of Eq. 15 over the
 * accepted Gaussians.  This tracer computes that product through the tree of
 * oracle_lbvh and gives the same T as the brute force whenever every Gaussian
 * that brute force accepts or flags lies in a box the ray meets:
 *   - leaf box of Gaussian j: the FP64 box of {m^2 <= K^2 + band_m2} (the
 *     support widened to the m^2 band), widened by 1e-9 of its half-extent and
 *     1e-12 (|mu| + 1) against rounding; internal boxes are unions;
 *   - a box counts when the ray meets it at some t >= -(2 band_t + 1e-12), so
 *     candidates with t* in the t band are reached too;
 *   - each candidate is evaluated by peak_m2 and the acceptance and band rules
 *     of oracle_trace.
 * Every candidate that oracle_trace accepts or flags has m^2 <= K^2 + band_m2
 * and t* >= -band_t, so it is visited.  The one difference: with t_min > 0 the
 * walk stops once the product of the accepted factors other than the
 * borderline ones (T_hi) is below t_min - band_T.  T is then 0 whatever
 * follows and whichever borderline factors are taken (the products only
 * fall), and a band flag that brute force would raise further along changes
 * nothing.  So T agrees with oracle_trace up to the order of the product, the
 * flags here are a subset of brute force's, and a ray flagged only by brute
 * force has T = 0; T_lo and T_hi are those of oracle_trace for a ray walked
 * to the end, and both below t_min - band_T for a stopped one.  Children are
 * visited nearer entry first so that the stop comes early.
 */
typedef struct {
    int64_t n;
    gauss64 *g;        /* original order */
    int32_t *left, *right;
    int32_t *leaf_id;  /* sorted position -> original index */
    double *ibox;      /* internal node boxes [n-1][6] */
    double *lbox;      /* leaf boxes [n][6], sorted order */
    double k_sigma, band_m2;
} orc_bvh;

static const double *node_box(const orc_bvh *b, uint32_t ref)
{
    return (ref & ORC_LEAF) ? b->lbox + 6 * (size_t)(ref & ~ORC_LEAF) : b->ibox + 6 * (size_t)ref;
}

/* Union boxes of internal nodes, children before parents (explicit stack). */
static void fill_internal_boxes(orc_bvh *b)
{
    int64_t m = b->n - 1;
    if (m <= 0) return;
    uint8_t *state = (uint8_t *)calloc((size_t)m, 1);
    int32_t *stk = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1));
    int64_t top = 0;
    stk[top++] = 0;
    while (top > 0) {
        int32_t i = stk[top - 1];
        uint32_t c[2] = {(uint32_t)b->left[i], (uint32_t)b->right[i]};
        if (!state[i]) {
            state[i] = 1;
            for (int k = 0; k < 2; ++k)
                if (!(c[k] & ORC_LEAF)) stk[top++] = (int32_t)c[k];
            continue;
        }
        --top;
        const double *x = node_box(b, c[0]), *y = node_box(b, c[1]);
        double *z = b->ibox + 6 * (size_t)i;
        for (int a = 0; a < 3; ++a) {
            z[a] = x[a] < y[a] ? x[a] : y[a];
            z[3 + a] = x[3 + a] > y[3 + a] ? x[3 + a] : y[3 + a];
        }
    }
    free(state);
    free(stk);
}

/*
 * Build the tracer over n Gaussians (FP64 inputs; the means must be float32
 * values, as the Morton codes are taken in float32).  Returns NULL on n < 0 or
 * allocation failure.  band_m2 is the m^2 band of oracle_trace the boxes must
 * cover.
 */
void *oracle_bvh_create(int64_t n, const double *mean, const double *scale, const double *quat,
                        const double *opac, double k_sigma, double band_m2)
{
    if (n < 0) return NULL;
    orc_bvh *b = (orc_bvh *)calloc(1, sizeof(orc_bvh));
    size_t n1 = (size_t)(n > 0 ? n : 1);
    b->n = n;
    b->k_sigma = k_sigma;
    b->band_m2 = band_m2;
    b->g = load_gaussians(n, mean, scale, quat, opac);
    b->left = (int32_t *)malloc(sizeof(int32_t) * n1);
    b->right = (int32_t *)malloc(sizeof(int32_t) * n1);
    b->leaf_id = (int32_t *)malloc(sizeof(int32_t) * n1);
    b->ibox = (double *)malloc(sizeof(double) * 6 * n1);
    b->lbox = (double *)malloc(sizeof(double) * 6 * n1);
    float *m32 = (float *)malloc(sizeof(float) * 3 * n1);
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * n1);
    int32_t *parent = (int32_t *)malloc(sizeof(int32_t) * 2 * n1);
    double *box = (double *)malloc(sizeof(double) * 6 * n1);
    for (int64_t i = 0; i < 3 * n; ++i) m32[i] = (float)mean[i];
    oracle_lbvh(n, m32, keys, b->left, b->right, parent);
    double kk = sqrt(k_sigma * k_sigma + band_m2);
    oracle_leaf_boxes(n, mean, scale, quat, opac, kk, 0.0, 0, box);
    for (int64_t p = 0; p < n; ++p) {
        int64_t j = (int64_t)(keys[p] & 0xffffffffu);
        b->leaf_id[p] = (int32_t)j;
        for (int a = 0; a < 3; ++a) {
            double c = mean[3 * j + a];
            double h = 0.5 * (box[6 * j + 3 + a] - box[6 * j + a]);
            double w = 1e-9 * h + 1e-12 * (fabs(c) + 1.0);
            b->lbox[6 * p + a] = box[6 * j + a] - w;
            b->lbox[6 * p + 3 + a] = box[6 * j + 3 + a] + w;
        }
    }
    fill_internal_boxes(b);
    free(m32);
    free(keys);
    free(parent);
    free(box);
    return b;
}

void oracle_bvh_destroy(void *h)
{
    orc_bvh *b = (orc_bvh *)h;
    if (!b) return;
    free(b->g);
    free(b->left);
    free(b->right);
    free(b->leaf_id);
    free(b->ibox);
    free(b->lbox);
    free(b);
}

/* Entry parameter of the ray into box bx on [t0, inf), or INFINITY if it
 * misses.  fmin/fmax drop the NaN of 0 * inf (a face through the origin on a
 * zero direction component), which can only keep a box, never lose one. */
static double slab64(const double *bx, const double o[3], const double inv[3], double t0)
{
    double lo = t0, hi = INFINITY;
    for (int a = 0; a < 3; ++a) {
        double ta = (bx[a] - o[a]) * inv[a], tb = (bx[3 + a] - o[a]) * inv[a];
        lo = fmax(lo, fmin(ta, tb));
        hi = fmin(hi, fmax(ta, tb));
    }
    return lo <= hi ? lo : INFINITY;
}

typedef struct {
    double alpha_min, t_min, band_m2, band_alpha, band_t, band_T;
} orc_rule;

/* One ray through the tree; returns T and writes T_exact (of the accepted
 * factors met before a stop), hits, flags, the bounds T_lo / T_hi of
 * oracle_trace and the box / Gaussian test counts.  The walk stops once even
 * T_hi (the product without the borderline candidates) is below
 * t_min - band_T: every subset then snaps to 0. */
static double bvh_ray(const orc_bvh *b, const orc_rule *u, const double ro[3], const double rd[3],
                      int64_t src, double *te_out, int32_t *hits_out, uint32_t *flags_out,
                      double *tlo_out, double *thi_out, int64_t *nbox, int64_t *ngauss)
{
    const double K2 = b->k_sigma * b->k_sigma;
    const double t0 = -(2.0 * u->band_t + 1e-12);
    const double stop = u->t_min > 0.0 ? u->t_min - u->band_T : -1.0;
    double inv[3];
    for (int a = 0; a < 3; ++a) inv[a] = 1.0 / rd[a];
    double tr = 1.0, tlo = 1.0, thi = 1.0;
    int32_t nh = 0;
    uint32_t fl = 0;
    uint32_t stk[130];
    int top = 0;
    if (b->n > 0) {
        uint32_t root = b->n == 1 ? ORC_LEAF : 0u;
        ++*nbox;
        if (slab64(node_box(b, root), ro, inv, t0) < INFINITY) stk[top++] = root;
    }
    while (top > 0 && thi >= stop) {
        uint32_t ref = stk[--top];
        if (ref & ORC_LEAF) {
            int64_t j = b->leaf_id[ref & ~ORC_LEAF];
            if (j == src) continue;
            ++*ngauss;
            double t;
            double m2 = peak_m2(&b->g[j], ro, rd, &t, NULL);
            double alpha = b->g[j].o * exp(-0.5 * m2);
            int ok_t = t > 0.0, ok_m = m2 <= K2, ok_a = alpha >= u->alpha_min;
            int near_t = fabs(t) <= u->band_t, near_m = fabs(m2 - K2) <= u->band_m2,
                near_a = fabs(alpha - u->alpha_min) <= u->band_alpha;
            int lo_t = ok_t || near_t, lo_m = ok_m || near_m, lo_a = ok_a || near_a;
            int border = 0;
            if (near_t && lo_m && lo_a) { fl |= ORC_FLAG_T; border = 1; }
            if (near_m && lo_t && lo_a) { fl |= ORC_FLAG_M2; border = 1; }
            if (near_a && lo_t && lo_m) { fl |= ORC_FLAG_ALPHA; border = 1; }
            if (ok_t && ok_m && ok_a) {
                tr *= (1.0 - alpha);
                ++nh;
            }
            if (border) {
                tlo *= (1.0 - alpha);
            } else if (ok_t && ok_m && ok_a) {
                tlo *= (1.0 - alpha);
                thi *= (1.0 - alpha);
            }
            continue;
        }
        uint32_t c[2] = {(uint32_t)b->left[ref], (uint32_t)b->right[ref]};
        double e[2];
        for (int k = 0; k < 2; ++k) e[k] = slab64(node_box(b, c[k]), ro, inv, t0);
        *nbox += 2;
        int near = e[1] < e[0] ? 1 : 0;
        /* the far child goes on the stack first; depth <= 64 keeps this bounded */
        if (e[1 - near] < INFINITY) stk[top++] = c[1 - near];
        if (e[near] < INFINITY) stk[top++] = c[near];
    }
    if (u->t_min > 0.0 && fabs(tr - u->t_min) <= u->band_T) fl |= ORC_FLAG_TMIN;
    *te_out = tr;
    *hits_out = nh;
    *flags_out = fl;
    *tlo_out = tlo;
    *thi_out = thi;
    return tr < u->t_min ? 0.0 : tr;
}

/*
 * Visibility of explicit rays through the tree (same arguments and outputs
 * as oracle_trace; T_exact, hits, flags, counts, T_lo, T_hi may be NULL).
 * counts[0..1] receive the total box and Gaussian tests.
 */
void oracle_bvh_trace(const void *h, int64_t n_rays, const double *ray_o, const double *ray_d,
                      const int32_t *ray_src, double alpha_min, double t_min, double band_alpha,
                      double band_t, double band_T, double *T, double *T_exact, int32_t *hits,
                      uint32_t *flags, int64_t *counts, double *T_lo, double *T_hi)
{
    const orc_bvh *b = (const orc_bvh *)h;
    orc_rule u = {alpha_min, t_min, b->band_m2, band_alpha, band_t, band_T};
    int64_t nb = 0, ng = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : nb, ng)
    for (int64_t r = 0; r < n_rays; ++r) {
        double ro[3] = {ray_o[3 * r], ray_o[3 * r + 1], ray_o[3 * r + 2]};
        double rd[3] = {ray_d[3 * r], ray_d[3 * r + 1], ray_d[3 * r + 2]};
        double te, tlo, thi;
        int32_t nh;
        uint32_t fl;
        T[r] = bvh_ray(b, &u, ro, rd, ray_src ? ray_src[r] : -1, &te, &nh, &fl, &tlo, &thi, &nb, &ng);
        if (T_lo) T_lo[r] = tlo;
        if (T_hi) T_hi[r] = thi;
        if (T_exact) T_exact[r] = te;
        if (hits) hits[r] = nh;
        if (flags) flags[r] = fl;
    }
    if (counts) { counts[0] = nb; counts[1] = ng; }
}

/*
 * Visibility of the direction-set rays (Sec. 4.2) through the tree, the rays
 * made as in oracle_dir_rays: ray id r = g*K + k, origin fl(mu_g + fl(eps d_k))
 * in float32, source g.  ids[m] lists the rays (NULL: all n*K in id order);
 * output i belongs to ray ids[i].
 */
void oracle_bvh_trace_dirs(const void *h, int32_t K, const float *dirs, float eps, const int64_t *ids,
                           int64_t m, double alpha_min, double t_min, double band_alpha, double band_t,
                           double band_T, double *T, double *T_exact, int32_t *hits, uint32_t *flags,
                           int64_t *counts, double *T_lo, double *T_hi)
{
    const orc_bvh *b = (const orc_bvh *)h;
    orc_rule u = {alpha_min, t_min, b->band_m2, band_alpha, band_t, band_T};
    int64_t nb = 0, ng = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : nb, ng)
    for (int64_t i = 0; i < m; ++i) {
        int64_t r = ids ? ids[i] : i;
        int64_t g = r / K;
        int32_t k = (int32_t)(r % K);
        double ro[3], rd[3];
        for (int a = 0; a < 3; ++a) {
            float d = dirs[3 * k + a];
            float off = eps * d;
            float o = (float)b->g[g].mu[a] + off;
            ro[a] = o;
            rd[a] = d;
        }
        double te, tlo, thi;
        int32_t nh;
        uint32_t fl;
        T[i] = bvh_ray(b, &u, ro, rd, g, &te, &nh, &fl, &tlo, &thi, &nb, &ng);
        if (T_lo) T_lo[i] = tlo;
        if (T_hi) T_hi[i] = thi;
        if (T_exact) T_exact[i] = te;
        if (hits) hits[i] = nh;
        if (flags) flags[i] = fl;
    }
    if (counts) { counts[0] = nb; counts[1] = ng; }
}

/* ------------------------------------------------------------------------ */
/* Visibility surrogate MLP (not in the paper)                               */
/* ------------------------------------------------------------------------ */

/* bf16 emulation switch: 1 (default) rounds where the GPU stores bf16; 0
 * makes the MLP exact FP64 (used to pin the backward by finite differences). */
static int g_bf16 = 1;
void oracle_mlp_set_bf16(int32_t on) { g_bf16 = on; }

/* Round to the nearest bfloat16 (ties to even) via float32, returned as double. */
static double bf16_round1(double x)
{
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) { /* inf / nan unchanged */
        return (double)f;
    }
    uint32_t lsb = (u >> 16) & 1u;
    u = (u + 0x7fffu + lsb) & 0xffff0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

static double bf16r(double x) { return g_bf16 ? bf16_round1(x) : x; }

void oracle_bf16_round(int64_t n, const double *x, double *y)
{
    for (int64_t i = 0; i < n; ++i) y[i] = bf16_round1(x[i]);
}

#define MLP_IN 80
#define MLP_H 128
#define MLP_FREQ 6

/*
 * Frequency encoding of one ray: six scalars (position normalised to [-1,1]
 * by the scene bounds, p_n = 2 (p - lo)/(hi - lo) - 1, then the direction),
 * each expanded to [x, sin(2^k pi x), cos(2^k pi x) for k = 0..5] (13 values),
 * 78 features, then two zeros: 80 inputs.
 */
static void encode(const float p[3], const float d[3], const float lo[3], const float hi[3], double out[MLP_IN])
{
    double x[6];
    for (int c = 0; c < 3; ++c) {
        double ext = (double)hi[c] - (double)lo[c];
        x[c] = ext > 0.0 ? 2.0 * ((double)p[c] - (double)lo[c]) / ext - 1.0 : 0.0;
        x[3 + c] = d[c];
    }
    int f = 0;
    for (int c = 0; c < 6; ++c) {
        out[f++] = x[c];
        for (int k = 0; k < MLP_FREQ; ++k) {
            double a = ldexp(M_PI, k) * x[c];
            out[f++] = sin(a);
            out[f++] = cos(a);
        }
    }
    out[f++] = 0.0;
    out[f++] = 0.0;
}

void oracle_mlp_encode(int64_t m, const float *pos, const float *dir, const float *lo, const float *hi, double *feat)
{
    for (int64_t i = 0; i < m; ++i) encode(pos + 3 * i, dir + 3 * i, lo, hi, feat + i * MLP_IN);
}

/* Parameter block layout (float32, as stored by the surrogate):
 *   W1[128][80], b1[128], W2[128][128], b2[128], W3[128][128], b3[128],
 *   W4[128][128], b4[128], w5[128], b5[1]. */
#define OFF_W1 0
#define OFF_B1 (OFF_W1 + MLP_H * MLP_IN)
#define OFF_W2 (OFF_B1 + MLP_H)
#define OFF_B2 (OFF_W2 + MLP_H * MLP_H)
#define OFF_W3 (OFF_B2 + MLP_H)
#define OFF_B3 (OFF_W3 + MLP_H * MLP_H)
#define OFF_W4 (OFF_B3 + MLP_H)
#define OFF_B4 (OFF_W4 + MLP_H * MLP_H)
#define OFF_W5 (OFF_B4 + MLP_H)
#define OFF_B5 (OFF_W5 + MLP_H)
#define MLP_NPARAM (OFF_B5 + 1)

int64_t oracle_mlp_nparam(void) { return MLP_NPARAM; }

/* Forward of one sample; acts[l] (l = 0..4) receive the bf16-rounded layer
 * inputs x_0 (encoding) .. x_4; returns the logit z5. */
static double mlp_fwd1(const float *P, const double *feat, double acts[5][MLP_H])
{
    static const int offW[4] = {OFF_W1, OFF_W2, OFF_W3, OFF_W4};
    static const int offB[4] = {OFF_B1, OFF_B2, OFF_B3, OFF_B4};
    for (int k = 0; k < MLP_IN; ++k) acts[0][k] = bf16r(feat[k]);
    for (int k = MLP_IN; k < MLP_H; ++k) acts[0][k] = 0.0;
    for (int l = 0; l < 4; ++l) {
        int kin = l == 0 ? MLP_IN : MLP_H;
        for (int o = 0; o < MLP_H; ++o) {
            double z = 0.0;
            for (int k = 0; k < kin; ++k) z += bf16r(P[offW[l] + o * kin + k]) * acts[l][k];
            z += (double)P[offB[l] + o];
            acts[l + 1][o] = bf16r(z > 0.0 ? z : 0.0);
        }
    }
    double z5 = (double)P[OFF_B5];
    for (int k = 0; k < MLP_H; ++k) z5 += (double)P[OFF_W5 + k] * acts[4][k];
    return z5;
}

/* p[i] = sigmoid(MLP(features of ray i)); logits optional. */
void oracle_mlp_forward(const float *P, int64_t m, const double *feat, double *p, double *logit)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        double acts[5][MLP_H];
        double z = mlp_fwd1(P, feat + i * MLP_IN, acts);
        if (logit) logit[i] = z;
        p[i] = 1.0 / (1.0 + exp(-z));
    }
}

/*
 * Visibility estimate of a network trained with weight w on the lit term of
 * the loss (below): the weighted loss is minimised by p = w T / (w T + 1 - T),
 * so T = p / (p + w (1 - p)) = 1 / (1 + w e^-z), z the logit.
 */
void oracle_mlp_visibility(const float *P, int64_t m, const double *feat, double w, double *T)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        double acts[5][MLP_H];
        double z = mlp_fwd1(P, feat + i * MLP_IN, acts);
        T[i] = 1.0 / (1.0 + w * exp(-z));
    }
}

/*
 * Mean binary cross-entropy against soft targets y, with weight w on the lit
 * term, L = -(1/m) sum_i [w y_i log p_i + (1 - y_i) log(1 - p_i)], and its
 * gradient for one minibatch of m samples.  dL/dz5 = (p (w y + 1 - y) - w y)/m
 * (= (p - y)/m for w = 1); for l = 4..1 the upstream
 * gradient of the pre-activation, dz_l = bf16(dx_l * [x_l > 0]), feeds
 * dW_l = sum_i dz_l x_{l-1}^T, db_l = sum_i dz_l and dx_{l-1} = bf16(W_l)^T dz_l
 * (FP64 sums).  grad has the parameter-block layout; returns the loss.
 */
double oracle_mlp_loss_grad(const float *P, int64_t m, const double *feat, const double *y, double w,
                            double *grad)
{
    static const int offW[4] = {OFF_W1, OFF_W2, OFF_W3, OFF_W4};
    static const int offB[4] = {OFF_B1, OFF_B2, OFF_B3, OFF_B4};
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    double *acc = (double *)calloc((size_t)nthreads * MLP_NPARAM, sizeof(double));
    double loss = 0.0;
#pragma omp parallel reduction(+ : loss)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *G = acc + (size_t)tid * MLP_NPARAM;
#pragma omp for schedule(static)
        for (int64_t i = 0; i < m; ++i) {
            double acts[5][MLP_H];
            double z = mlp_fwd1(P, feat + i * MLP_IN, acts);
            double p = 1.0 / (1.0 + exp(-z));
            double yi = y[i];
            /* log(1+e^-z) and log(1+e^z), stably */
            double sp_neg = (z > 0 ? 0.0 : -z) + log1p(exp(-fabs(z)));
            double sp_pos = (z > 0 ? z : 0.0) + log1p(exp(-fabs(z)));
            loss += (w * yi * sp_neg + (1.0 - yi) * sp_pos) / (double)m;
            double dz5 = (p * (w * yi + 1.0 - yi) - w * yi) / (double)m;
            G[OFF_B5] += dz5;
            double dx[MLP_H];
            for (int k = 0; k < MLP_H; ++k) {
                G[OFF_W5 + k] += dz5 * acts[4][k];
                dx[k] = dz5 * (double)P[OFF_W5 + k];
            }
            for (int l = 3; l >= 0; --l) {
                int kin = l == 0 ? MLP_IN : MLP_H;
                double dz[MLP_H];
                for (int o = 0; o < MLP_H; ++o) dz[o] = bf16r(acts[l + 1][o] > 0.0 ? dx[o] : 0.0);
                for (int o = 0; o < MLP_H; ++o) {
                    G[offB[l] + o] += dz[o];
                    for (int k = 0; k < kin; ++k) G[offW[l] + o * kin + k] += dz[o] * acts[l][k];
                }
                if (l > 0) {
                    for (int k = 0; k < kin; ++k) {
                        double s = 0.0;
                        for (int o = 0; o < MLP_H; ++o) s += bf16r(P[offW[l] + o * kin + k]) * dz[o];
                        dx[k] = s;
                    }
                }
            }
        }
    }
    for (int64_t q = 0; q < MLP_NPARAM; ++q) {
        double s = 0.0;
        for (int t = 0; t < nthreads; ++t) s += acc[(size_t)t * MLP_NPARAM + (size_t)q];
        grad[q] = s;
    }
    free(acc);
    return loss;
}

/* One Adam step (Kingma & Ba 2015) with bias correction, step count t >= 1. */
void oracle_adam_step(int64_t n, double *w, const double *g, double *mo, double *vo, int64_t t,
                      double lr, double b1, double b2, double eps)
{
    double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
    for (int64_t i = 0; i < n; ++i) {
        mo[i] = b1 * mo[i] + (1.0 - b1) * g[i];
        vo[i] = b2 * vo[i] + (1.0 - b2) * g[i] * g[i];
        double mh = mo[i] / c1, vh = vo[i] / c2;
        w[i] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* ------------------------------------------------------------------------ */
/* Hemisphere direction sets and the per-Gaussian PBR colour (Sec. 3.3)      */
/* ------------------------------------------------------------------------ */

/*
 * Sec. 3.3 samples N_s incident directions per Gaussian over the hemisphere
 * about its normal n (Fibonacci sampling) and Sec. 4.2 precomputes the
 * visibility of those directions.  Ray id r = g*K + k of Gaussian g uses the
 * local direction hemi[k] (z along the normal) in an orthonormal frame
 * (t1, t2, n) built from the normal with the branchless construction of
 * Duff et al. 2017 ("Building an orthonormal basis, revisited").  All in
 * float32 with separately rounded operations, in this order:
 *   s = (nx*nx + ny*ny) + nz*nz;  l = sqrt(s);  n = (nx/l, ny/l, nz/l)
 *   sg = copysign(1, nz);  a = -1 / (sg + nz);  b = (nx*ny)*a
 *   t1 = (1 + ((sg*nx)*nx)*a,  sg*b,  -(sg*nx))
 *   t2 = (b,  sg + (ny*ny)*a,  -ny)
 *   d_c = (h_x*t1_c + h_y*t2_c) + h_z*n_c
 * and the origin fl(mu + fl(eps*d)) as in oracle_dir_rays.
 */
static void hemi_frame(const float *nin, float t1[3], float t2[3], float n[3])
{
    float s = nin[0] * nin[0] + nin[1] * nin[1];
    s = s + nin[2] * nin[2];
    float l = sqrtf(s);
    n[0] = nin[0] / l;
    n[1] = nin[1] / l;
    n[2] = nin[2] / l;
    float sg = copysignf(1.0f, n[2]);
    float a = -1.0f / (sg + n[2]);
    float b = (n[0] * n[1]) * a;
    t1[0] = 1.0f + ((sg * n[0]) * n[0]) * a;
    t1[1] = sg * b;
    t1[2] = -(sg * n[0]);
    t2[0] = b;
    t2[1] = sg + (n[1] * n[1]) * a;
    t2[2] = -n[1];
}

static void hemi_dir(const float *nin, const float *h, float d[3])
{
    float t1[3], t2[3], n[3];
    hemi_frame(nin, t1, t2, n);
    for (int c = 0; c < 3; ++c) {
        float x = h[0] * t1[c] + h[1] * t2[c];
        d[c] = x + h[2] * n[c];
    }
}

void oracle_hemi_rays(int64_t n, const float *mean, const float *normals, int32_t K, const float *hemi,
                      float eps, const int64_t *ids, int64_t m, float *ray_o, float *ray_d, int32_t *ray_src)
{
    (void)n;
    for (int64_t i = 0; i < m; ++i) {
        int64_t r = ids[i];
        int64_t g = r / K;
        int32_t k = (int32_t)(r % K);
        float d[3];
        hemi_dir(normals + 3 * g, hemi + 3 * k, d);
        for (int c = 0; c < 3; ++c) {
            float off = eps * d[c];
            ray_o[3 * i + c] = mean[3 * g + c] + off;
            ray_d[3 * i + c] = d[c];
        }
        ray_src[i] = (int32_t)g;
    }
}

/*
 * Simplified Disney BRDF of Sec. 3.3 (Eq. 9): f = f_d + f_s with f_d = b/pi
 * and the microfacet specular term f_s = D F G / (4 (n.wi)(n.wo)).  Readings
 * (the paper names D, F, G without formulas):
 *   h  = (wi + wo)/|wi + wo|  (the half vector, normalised; f_s = 0 if wi = -wo);
 *   D  = GGX / Trowbridge-Reitz with alpha = r^2:
 *        alpha^2 / (pi ((n.h)^2 (alpha^2 - 1) + 1)^2);
 *   F  = Schlick with F0 = 0.04 (the model has no metallic parameter):
 *        F0 + (1 - F0)(1 - max(wo.h, 0))^5;
 *   G  = Smith with Schlick-GGX, k = (r + 1)^2 / 8:
 *        G1(x) = x / (x (1 - k) + k),  G = G1(n.wi) G1(n.wo);
 *   the factor 4 of the microfacet model, which the printed Eq. 9 omits
 *   (without it the specular lobe reflects more energy than it receives);
 *   n.wi and n.wo clamped at 0; r clamped to [0.04, 1].
 * G1(x)/x = 1/(x(1-k)+k) is used, so f_s stays finite at grazing angles.
 * Inputs FP64 unit vectors.  fs_terms (may be NULL) gets D, F, G.
 */
#define PBR_F0 0.04
#define PBR_RMIN 0.04

static double spec_term(const double n[3], const double wi[3], const double wo[3], double r, double *Dout,
                        double *Fout, double *Gout)
{
    if (r < PBR_RMIN) r = PBR_RMIN;
    if (r > 1.0) r = 1.0;
    double nl = n[0] * wi[0] + n[1] * wi[1] + n[2] * wi[2];
    double nv = n[0] * wo[0] + n[1] * wo[1] + n[2] * wo[2];
    if (nl < 0.0) nl = 0.0;
    if (nv < 0.0) nv = 0.0;
    double hv[3] = {wi[0] + wo[0], wi[1] + wo[1], wi[2] + wo[2]};
    double hl = sqrt(hv[0] * hv[0] + hv[1] * hv[1] + hv[2] * hv[2]);
    if (!(hl > 0.0)) {
        if (Dout) *Dout = 0.0;
        if (Fout) *Fout = 0.0;
        if (Gout) *Gout = 0.0;
        return 0.0;
    }
    for (int c = 0; c < 3; ++c) hv[c] /= hl;
    double nh = n[0] * hv[0] + n[1] * hv[1] + n[2] * hv[2];
    double vh = wo[0] * hv[0] + wo[1] * hv[1] + wo[2] * hv[2];
    if (vh < 0.0) vh = 0.0;
    double al = r * r, a2 = al * al;
    double q = nh * nh * (a2 - 1.0) + 1.0;
    double D = a2 / (M_PI * q * q);
    double F = PBR_F0 + (1.0 - PBR_F0) * pow(1.0 - vh, 5.0);
    double k = (r + 1.0) * (r + 1.0) / 8.0;
    double gl = 1.0 / (nl * (1.0 - k) + k), gv = 1.0 / (nv * (1.0 - k) + k);  /* G1(x)/x */
    if (Dout) *Dout = D;
    if (Fout) *Fout = F;
    if (Gout) *Gout = (nl * gl) * (nv * gv);
    return D * F * gl * gv / 4.0;
}

void oracle_brdf_spec(int64_t m, const double *n, const double *wi, const double *wo, const double *rough,
                      double *fs, double *terms)
{
    for (int64_t i = 0; i < m; ++i) {
        double D, F, G;
        fs[i] = spec_term(n + 3 * i, wi + 3 * i, wo + 3 * i, rough[i], &D, &F, &G);
        if (terms) {
            terms[3 * i] = D;
            terms[3 * i + 1] = F;
            terms[3 * i + 2] = G;
        }
    }
}

/*
 * Indirect light of Sec. 3.3 ("3-level SH"): real spherical harmonics of
 * degree 0..2 (9 functions) in the usual real basis, e.g. as in 3D Gaussian
 * splatting: Y0 = c0; Y1..3 = -c1 y, c1 z, -c1 x; Y4..8 = c2a xy, -c2a yz,
 * c2b (2z^2 - x^2 - y^2), -c2a xz, c2c (x^2 - y^2), with c0 = 1/(2 sqrt(pi)),
 * c1 = sqrt(3/(4 pi)), c2a = sqrt(15/(4 pi)), c2b = sqrt(5/(16 pi)),
 * c2c = sqrt(15/(16 pi)).
 */
static void sh9(const double w[3], double Y[9])
{
    const double c0 = 0.5 / sqrt(M_PI), c1 = sqrt(3.0 / (4.0 * M_PI)), c2a = sqrt(15.0 / (4.0 * M_PI)),
                 c2b = sqrt(5.0 / (16.0 * M_PI)), c2c = sqrt(15.0 / (16.0 * M_PI));
    double x = w[0], y = w[1], z = w[2];
    Y[0] = c0;
    Y[1] = -c1 * y;
    Y[2] = c1 * z;
    Y[3] = -c1 * x;
    Y[4] = c2a * x * y;
    Y[5] = -c2a * y * z;
    Y[6] = c2b * (2.0 * z * z - x * x - y * y);
    Y[7] = -c2a * x * z;
    Y[8] = c2c * (x * x - y * y);
}

void oracle_sh_basis(int64_t m, const double *w, double *Y)
{
    for (int64_t i = 0; i < m; ++i) sh9(w + 3 * i, Y + 9 * i);
}

/*
 * Direct light of Sec. 3.3: a global h x w environment map (16 x 32 in the
 * paper), RGB, equirectangular: row i covers polar angles [i pi/h, (i+1) pi/h]
 * from +z, column j azimuths [2 pi j/w, 2 pi (j+1)/w].  Reading: bilinear
 * interpolation between pixel centres (continuous in the direction), wrapping
 * in azimuth and clamped to the first and last rows in polar angle.
 */
static void env_bilinear(int32_t h, int32_t w, const double *env, const double d[3], double L[3])
{
    double z = d[2];
    if (z > 1.0) z = 1.0;
    if (z < -1.0) z = -1.0;
    double th = acos(z);
    double ph = atan2(d[1], d[0]);
    if (ph < 0.0) ph += 2.0 * M_PI;
    double v = th / M_PI * h - 0.5, u = ph / (2.0 * M_PI) * w - 0.5;
    double fv = floor(v), fu = floor(u);
    double bv = v - fv, bu = u - fu;
    int64_t i0 = (int64_t)fv, j0 = (int64_t)fu;
    int64_t i1 = i0 + 1, j1 = j0 + 1;
    if (i0 < 0) i0 = 0;
    if (i1 < 0) i1 = 0;
    if (i0 > h - 1) i0 = h - 1;
    if (i1 > h - 1) i1 = h - 1;
    j0 = ((j0 % w) + w) % w;
    j1 = ((j1 % w) + w) % w;
    for (int c = 0; c < 3; ++c) {
        double a = env[(i0 * w + j0) * 3 + c] * (1.0 - bu) + env[(i0 * w + j1) * 3 + c] * bu;
        double b = env[(i1 * w + j0) * 3 + c] * (1.0 - bu) + env[(i1 * w + j1) * 3 + c] * bu;
        L[c] = a * (1.0 - bv) + b * bv;
    }
}

void oracle_env_lookup(int32_t h, int32_t w, const double *env, int64_t m, const double *dirs, double *L)
{
    for (int64_t i = 0; i < m; ++i) env_bilinear(h, w, env, dirs + 3 * i, L + 3 * i);
}

/*
 * Per-Gaussian PBR colour, Eq. 10: for Gaussian g with normal n (the float32
 * normal normalised in FP64), albedo b, roughness r, SH coefficients
 * sh[g][9][3] (NULL: no indirect light) and view direction
 * wo = (cam - mu)/|cam - mu|,
 *   c'_c = sum_k (b_c/pi + f_s(wo, wi_k)) L_c(wi_k) max(n.wi_k, 0) (2 pi / K)
 *   L_c(wi) = V[g,k] L_direct,c(wi) + max(0, sum_j sh[g][j][c] Y_j(wi))
 * (Eq. 8: visibility times direct light plus indirect light; the solid angle
 * of one of K directions on the hemisphere is 2 pi / K; reading: the
 * indirect light is clamped at 0).  wi_k is ray k of Gaussian g from
 * oracle_hemi_rays (float32, widened).  V[g*K + k] is the traced visibility.
 */
void oracle_pbr(int64_t n, const float *mean, const float *normals, const float *albedo, const float *rough,
                const float *sh, int32_t K, const float *hemi, const double *V, int32_t h, int32_t w,
                const double *env, const double *cam, double *rgb)
{
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t g = 0; g < n; ++g) {
        double nn[3] = {normals[3 * g], normals[3 * g + 1], normals[3 * g + 2]};
        double l = sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
        for (int c = 0; c < 3; ++c) nn[c] /= l;
        double wo[3] = {cam[0] - mean[3 * g], cam[1] - mean[3 * g + 1], cam[2] - mean[3 * g + 2]};
        double lo = sqrt(wo[0] * wo[0] + wo[1] * wo[1] + wo[2] * wo[2]);
        for (int c = 0; c < 3; ++c) wo[c] /= lo;
        double acc[3] = {0.0, 0.0, 0.0};
        for (int32_t k = 0; k < K; ++k) {
            float df[3];
            hemi_dir(normals + 3 * g, hemi + 3 * k, df);
            double wi[3] = {df[0], df[1], df[2]};
            double nl = nn[0] * wi[0] + nn[1] * wi[1] + nn[2] * wi[2];
            if (nl < 0.0) nl = 0.0;
            double fs = spec_term(nn, wi, wo, rough[g], NULL, NULL, NULL);
            double Ld[3], Y[9];
            env_bilinear(h, w, env, wi, Ld);
            if (sh) sh9(wi, Y);
            for (int c = 0; c < 3; ++c) {
                double Li = V[g * K + k] * Ld[c];
                if (sh) {
                    double s = 0.0;
                    for (int j = 0; j < 9; ++j) s += sh[(g * 9 + j) * 3 + c] * Y[j];
                    if (s > 0.0) Li += s;
                }
                acc[c] += (albedo[3 * g + c] / M_PI + fs) * Li * nl;
            }
        }
        for (int c = 0; c < 3; ++c) rgb[3 * g + c] = acc[c] * (2.0 * M_PI / K);
    }
}
