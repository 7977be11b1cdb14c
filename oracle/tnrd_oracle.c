/*
 * FP64 CPU oracle for the TRDMD despeckling stage -- TEST INFRASTRUCTURE ONLY.
 * See tnrd_oracle.h for the method, the readings of the paper it follows, and
 * who may call it.  Every function is the plain definition written out: no
 * blocking, no window truncation of the RBF sum, no recurrences, no FFT.
 * OpenMP (when enabled) only splits independent outputs between threads; the
 * arithmetic of each output is the same as in a serial run.
 */
#include "tnrd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

long orc_sym(long i, long n)
{
    long m = i % (2 * n);
    if (m < 0) m += 2 * n;
    return m < n ? m : 2 * n - 1 - m;
}

/* Eq. diffusion: k * u, "2D convolution of the image u with the filter k",
 * read as true convolution over the symmetric-padded image. */
void orc_conv(const double* u, int H, int W, const double* k, int ks, double* z)
{
    const int r = ks / 2;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            double s = 0.0;
            for (int a = 0; a < ks; ++a) {
                const long yy = orc_sym(y + r - a, H);
                for (int b = 0; b < ks; ++b) {
                    const long xx = orc_sym(x + r - b, W);
                    s += k[a * ks + b] * u[yy * W + xx];
                }
            }
            z[(long)y * W + x] = s;
        }
    }
}

/* K^T (Eq. derv1-1, "careful boundary handling"): the literal transpose of
 * orc_conv, every product scattered to the pixel it was gathered from. */
void orc_conv_adj(const double* v, int H, int W, const double* k, int ks, double* out)
{
    const int r = ks / 2;
    memset(out, 0, sizeof(double) * (size_t)H * (size_t)W);
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            const double vv = v[(long)y * W + x];
            for (int a = 0; a < ks; ++a) {
                const long yy = orc_sym(y + r - a, H);
                for (int b = 0; b < ks; ++b) {
                    const long xx = orc_sym(x + r - b, W);
                    out[yy * W + xx] += k[a * ks + b] * vv;
                }
            }
        }
    }
}

double orc_rbf(double z, int j, double mu0, double delta, double gamma)
{
    const double d = z - (mu0 + delta * j);
    return exp(-(d * d) / (2.0 * gamma * gamma));
}

double orc_phi(double z, const double* w, int nrbf, double mu0, double delta, double gamma)
{
    double s = 0.0;
    for (int j = 0; j < nrbf; ++j) s += w[j] * orc_rbf(z, j, mu0, delta, gamma);
    return s;
}

double orc_dphi(double z, const double* w, int nrbf, double mu0, double delta, double gamma)
{
    double s = 0.0;
    for (int j = 0; j < nrbf; ++j) {
        const double d = z - (mu0 + delta * j);
        s += w[j] * orc_rbf(z, j, mu0, delta, gamma) * (-d / (gamma * gamma));
    }
    return s;
}

void orc_phi_vec(const double* z, long n, const double* w, int nrbf,
                 double mu0, double delta, double gamma, double* out)
{
#pragma omp parallel for schedule(static)
    for (long p = 0; p < n; ++p) out[p] = orc_phi(z[p], w, nrbf, mu0, delta, gamma);
}

void orc_dphi_vec(const double* z, long n, const double* w, int nrbf,
                  double mu0, double delta, double gamma, double* out)
{
#pragma omp parallel for schedule(static)
    for (long p = 0; p < n; ++p) out[p] = orc_dphi(z[p], w, nrbf, mu0, delta, gamma);
}

void orc_diffusion(const double* u, int H, int W, const double* k, const double* w,
                   int nk, int ks, int nrbf, double mu0, double delta, double gamma,
                   double* out)
{
    const long n = (long)H * W;
    double* z = (double*)malloc(sizeof(double) * n);
    double* v = (double*)malloc(sizeof(double) * n);
    double* kt = (double*)malloc(sizeof(double) * n);
    memset(out, 0, sizeof(double) * n);
    for (int i = 0; i < nk; ++i) {
        orc_conv(u, H, W, k + (long)i * ks * ks, ks, z);
        orc_phi_vec(z, n, w + (long)i * nrbf, nrbf, mu0, delta, gamma, v);
        orc_conv_adj(v, H, W, k + (long)i * ks * ks, ks, kt);
        for (long p = 0; p < n; ++p) out[p] += kt[p];
    }
    free(z);
    free(v);
    free(kt);
}

/* Eq. subproblemGIdiv.  For u~ < 0 the same root is written as
 * 4 lam f^2 / (S - u~) (multiply numerator and denominator by S - u~), which
 * avoids cancelling two nearly equal numbers; the two forms are identical. */
double orc_prox(double ut, double f, double lam)
{
    const double a = 1.0 + 2.0 * lam;
    const double S = sqrt(ut * ut + 8.0 * a * lam * f * f);
    if (ut >= 0.0) return (ut + S) / (2.0 * a);
    if (S - ut == 0.0) return 0.0;
    return 4.0 * lam * f * f / (S - ut);
}

void orc_prox_vec(const double* ut, const double* f, long n, double lam, double* u)
{
    for (long p = 0; p < n; ++p) u[p] = orc_prox(ut[p], f[p], lam);
}

/* Eq. derv2: y = (1 + u~/S) / (2 (1 + 2 lam)). */
double orc_prox_du(double ut, double f, double lam)
{
    const double a = 1.0 + 2.0 * lam;
    const double S = sqrt(ut * ut + 8.0 * a * lam * f * f);
    const double r = (S > 0.0) ? ut / S : 0.0;
    return (1.0 + r) / (2.0 * a);
}

/* Eq. derv4: x = (2 f^2 + 8 lam f^2) / ((1 + 2 lam) S) - (u~ + S) / (1 + 2 lam)^2. */
double orc_prox_dlam(double ut, double f, double lam)
{
    const double a = 1.0 + 2.0 * lam;
    const double S = sqrt(ut * ut + 8.0 * a * lam * f * f);
    const double t1 = (S > 0.0) ? (2.0 * f * f + 8.0 * lam * f * f) / (a * S) : 0.0;
    return t1 - (ut + S) / (a * a);
}

/* Reaction term psi(u) of the explicit data-term steps and its derivative:
 *   ORC_GAUSS: psi = lam (u - f),                 psi' = lam
 *   ORC_PROJ:  psi = (lam / u) (1 - f^2 / u^2),   psi' = -lam / u^2 + 3 lam f^2 / u^4
 * (the gradient of lam/2 |u - f|^2, resp. of lam <log u + f^2 / (2 u^2), 1>). */
static double orc_psi(int mode, double u, double f, double lam)
{
    if (mode == ORC_GAUSS) return lam * (u - f);
    if (mode == ORC_PROJ) return (lam / u) * (1.0 - (f * f) / (u * u));
    return 0.0;
}

static double orc_dpsi(int mode, double u, double f, double lam)
{
    if (mode == ORC_GAUSS) return lam;
    if (mode == ORC_PROJ) return -lam / (u * u) + 3.0 * lam * f * f / (u * u * u * u);
    return 0.0;
}

void orc_stage_mode(const double* u_prev, const double* f, int H, int W, int t,
                    const double* k, const double* w, const double* lam,
                    int nk, int ks, int nrbf, double mu0, double delta, double gamma,
                    int mode, double c, double* u_next, double* ut_out)
{
    const long n = (long)H * W;
    double* g = (double*)malloc(sizeof(double) * n);
    double* ut = (double*)malloc(sizeof(double) * n);
    orc_diffusion(u_prev, H, W, k + (long)t * nk * ks * ks, w + (long)t * nk * nrbf,
                  nk, ks, nrbf, mu0, delta, gamma, g);
    for (long p = 0; p < n; ++p)
        ut[p] = u_prev[p] - g[p] - orc_psi(mode, u_prev[p], f[p], lam[t]);
    if (mode == ORC_IDIV) {
        orc_prox_vec(ut, f, n, lam[t], u_next);
    } else if (mode == ORC_GAUSS) {
        memcpy(u_next, ut, sizeof(double) * n);
    } else {
        for (long p = 0; p < n; ++p) u_next[p] = ut[p] > c ? ut[p] : c;
    }
    if (ut_out) memcpy(ut_out, ut, sizeof(double) * n);
    free(g);
    free(ut);
}

void orc_stage(const double* u_prev, const double* f, int H, int W, int t,
               const double* k, const double* w, const double* lam,
               int nk, int ks, int nrbf, double mu0, double delta, double gamma,
               double* u_next, double* ut_out)
{
    orc_stage_mode(u_prev, f, H, W, t, k, w, lam, nk, ks, nrbf, mu0, delta, gamma,
                   ORC_IDIV, 0.0, u_next, ut_out);
}

void orc_forward_mode(const double* f, int H, int W, int T,
                      const double* k, const double* w, const double* lam,
                      int nk, int ks, int nrbf, double mu0, double delta, double gamma,
                      int mode, double c, double* u_all)
{
    const long n = (long)H * W;
    memcpy(u_all, f, sizeof(double) * n);
    for (int t = 0; t < T; ++t)
        orc_stage_mode(u_all + t * n, f, H, W, t, k, w, lam, nk, ks, nrbf, mu0, delta, gamma,
                       mode, c, u_all + (t + 1) * n, NULL);
}

void orc_forward(const double* f, int H, int W, int T,
                 const double* k, const double* w, const double* lam,
                 int nk, int ks, int nrbf, double mu0, double delta, double gamma,
                 double* u_all)
{
    orc_forward_mode(f, H, W, T, k, w, lam, nk, ks, nrbf, mu0, delta, gamma, ORC_IDIV, 0.0,
                     u_all);
}

/* Back-propagation through the cascade (Eq. iterstep), stage by stage from T
 * down to 1.  For stage t with e = dL/du_t, u~ = u - diffusion(u) - psi(u) and
 * u_t = P(u~) (P the prox, the identity or max(., c)):
 *   s      = P'(u~): y of Eq. derv2 / 1 / [u~ > c]
 *   d      = s .* e                                       (Eqs. derv1, derv2)
 *   dlam_t = sum_p e_p du_t/dlam: x of Eq. derv4 / -(u - f) d / -(psi/lam) d
 *   b_i    = K_i d
 *   dw_ij  = -sum_p b_i(p) G_j(z_i(p))                    (phi_i linear in w_i)
 *   c_i    = -phi_i'(z_i) .* b_i
 *   dk_i   = sum_p c_i(p) * dz_i(p)/dk_i - v_i(p) * d(K_i d)(p)/dk_i ... both
 *            written out as the shifted products of the padded images
 *   dL/du_{t-1} = (1 - psi'(u)) d + sum_i K_i^T c_i       (Eq. derv1-1)
 */
void orc_backward_mode(const double* f, int H, int W, int T,
                       const double* k, const double* w, const double* lam,
                       int nk, int ks, int nrbf, double mu0, double delta, double gamma,
                       int mode, double cproj, const double* u_all, const double* e_T,
                       double* e_0, double* gk, double* gw, double* glam)
{
    const long n = (long)H * W;
    const int r = ks / 2;
    double* e = (double*)malloc(sizeof(double) * n);
    double* e_prev = (double*)malloc(sizeof(double) * n);
    double* ut = (double*)malloc(sizeof(double) * n);
    double* unext = (double*)malloc(sizeof(double) * n);
    double* d = (double*)malloc(sizeof(double) * n);
    double* z = (double*)malloc(sizeof(double) * n);
    double* v = (double*)malloc(sizeof(double) * n);
    double* b = (double*)malloc(sizeof(double) * n);
    double* c = (double*)malloc(sizeof(double) * n);
    double* kt = (double*)malloc(sizeof(double) * n);
    memcpy(e, e_T, sizeof(double) * n);

    for (int t = T - 1; t >= 0; --t) {
        const double* u = u_all + t * n;
        const double* kt_ = k + (long)t * nk * ks * ks;
        const double* wt_ = w + (long)t * nk * nrbf;
        /* recompute u~ of this stage */
        orc_stage_mode(u, f, H, W, t, k, w, lam, nk, ks, nrbf, mu0, delta, gamma, mode, cproj,
                       unext, ut);
        double sl = 0.0;
        for (long p = 0; p < n; ++p) {
            if (mode == ORC_IDIV) {
                d[p] = orc_prox_du(ut[p], f[p], lam[t]) * e[p];
                sl += orc_prox_dlam(ut[p], f[p], lam[t]) * e[p];
            } else {
                const double s = (mode == ORC_GAUSS) ? 1.0 : (ut[p] > cproj ? 1.0 : 0.0);
                d[p] = s * e[p];
                /* psi is linear in lam: du~/dlam = -psi / lam */
                sl += -(orc_psi(mode, u[p], f[p], 1.0)) * d[p];
            }
            e_prev[p] = (1.0 - orc_dpsi(mode, u[p], f[p], lam[t])) * d[p];
        }
        glam[t] = sl;
        for (int i = 0; i < nk; ++i) {
            const double* ki = kt_ + (long)i * ks * ks;
            const double* wi = wt_ + (long)i * nrbf;
            orc_conv(u, H, W, ki, ks, z);
            orc_phi_vec(z, n, wi, nrbf, mu0, delta, gamma, v);
            orc_conv(d, H, W, ki, ks, b);
            for (int j = 0; j < nrbf; ++j) {
                double s = 0.0;
                for (long p = 0; p < n; ++p) s += b[p] * orc_rbf(z[p], j, mu0, delta, gamma);
                gw[((long)t * nk + i) * nrbf + j] = -s;
            }
            orc_dphi_vec(z, n, wi, nrbf, mu0, delta, gamma, c);
            for (long p = 0; p < n; ++p) c[p] = -c[p] * b[p];
            for (int a = 0; a < ks; ++a) {
                for (int bb = 0; bb < ks; ++bb) {
                    double s = 0.0;
                    for (int y = 0; y < H; ++y) {
                        const long yy = orc_sym(y + r - a, H);
                        for (int x = 0; x < W; ++x) {
                            const long xx = orc_sym(x + r - bb, W);
                            const long p = (long)y * W + x;
                            s += c[p] * u[yy * W + xx] - v[p] * d[yy * W + xx];
                        }
                    }
                    gk[(((long)t * nk + i) * ks + a) * ks + bb] = s;
                }
            }
            orc_conv_adj(c, H, W, ki, ks, kt);
            for (long p = 0; p < n; ++p) e_prev[p] += kt[p];
        }
        memcpy(e, e_prev, sizeof(double) * n);
    }
    if (e_0) memcpy(e_0, e, sizeof(double) * n);
    free(e); free(e_prev); free(ut); free(unext); free(d); free(z); free(v);
    free(b); free(c); free(kt);
}

void orc_backward(const double* f, int H, int W, int T,
                  const double* k, const double* w, const double* lam,
                  int nk, int ks, int nrbf, double mu0, double delta, double gamma,
                  const double* u_all, const double* e_T,
                  double* e_0, double* gk, double* gw, double* glam)
{
    orc_backward_mode(f, H, W, T, k, w, lam, nk, ks, nrbf, mu0, delta, gamma, ORC_IDIV, 0.0,
                      u_all, e_T, e_0, gk, gw, glam);
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
