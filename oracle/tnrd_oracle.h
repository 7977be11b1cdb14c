/*
 * FP64 CPU oracle for one TRDMD despeckling stage and its T-stage cascade.
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the plain, slow, obviously correct
 * restatement of the method that the CUDA path is checked against.  Only the
 * test-suite, the smoke check and the benchmark's CPU-baseline leg may load it;
 * the product path never calls it and shares no code with it.
 *
 * Method (Feng & Chen, "Speckle Reduction with Trained Nonlinear Diffusion
 * Filtering"):
 *   stage (Eq. diffusionprocessfinal, Sec. 3.1):
 *     u~_t = u_{t-1} - sum_i K_i^T phi_i(K_i u_{t-1})
 *     u_t  = (u~ + sqrt(u~^2 + 8 (1+2 lam) lam f^2)) / (2 (1+2 lam))   (Eq. subproblemGIdiv)
 *   cascade (Eq. diffusion): u_0 = f, t = 1..T.
 *   gradients (Sec. 3.2, Eqs. derv1, derv1-1, derv2, derv4, iterstep).
 *   the same stage with the TNRD Gaussian-denoising reaction term (Sec. 2.2.1)
 *   and with the explicit data-term step plus projection (Eq. diffusion_backP).
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - "*" is true 2-D convolution; boundary is half-sample symmetric padding
 *     and K^T is the exact matrix transpose of the padded convolution.
 *   - phi_i(z) = sum_j w_ij exp(-(z - mu_j)^2 / (2 gamma^2)), mu_j = mu0 + j*delta.
 *   - u_0 = f.
 *   - where S = sqrt(u~^2 + 8 a lam f^2) is 0 (only if f = 0 or lam = 0 with
 *     u~ = 0), the ratios u~/S and f^2/S in Eqs. derv2/derv4 are taken as 0.
 *
 * All arrays are dense row-major doubles with no padding.  Parameters of a
 * T-stage model: k [T][nk][ks][ks], w [T][nk][nrbf], lam [T].
 */
#ifndef TNRD_ORACLE_H
#define TNRD_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Half-sample symmetric index into [0, n): ... 1 0 | 0 1 ... n-1 | n-1 n-2 ... */
long orc_sym(long i, long n);

/* z = K u : z(y,x) = sum_{a,b} k[a][b] u(sym(y+r-a), sym(x+r-b)), r = ks/2. */
void orc_conv(const double* u, int H, int W, const double* k, int ks, double* z);

/* out = K^T v by scatter: out[sym(y+r-a)][sym(x+r-b)] += k[a][b] v(y,x). */
void orc_conv_adj(const double* v, int H, int W, const double* k, int ks, double* out);

/* Gaussian RBF G_j(z) = exp(-(z - mu_j)^2 / (2 gamma^2)). */
double orc_rbf(double z, int j, double mu0, double delta, double gamma);
/* phi(z) = sum_j w_j G_j(z), all nrbf terms. */
double orc_phi(double z, const double* w, int nrbf, double mu0, double delta, double gamma);
/* phi'(z) = sum_j w_j G_j(z) * (-(z - mu_j) / gamma^2). */
double orc_dphi(double z, const double* w, int nrbf, double mu0, double delta, double gamma);
void orc_phi_vec(const double* z, long n, const double* w, int nrbf,
                 double mu0, double delta, double gamma, double* out);
void orc_dphi_vec(const double* z, long n, const double* w, int nrbf,
                  double mu0, double delta, double gamma, double* out);

/* Diffusion force sum_i K_i^T phi_i(K_i u) of one stage (nk filters). */
void orc_diffusion(const double* u, int H, int W, const double* k, const double* w,
                   int nk, int ks, int nrbf, double mu0, double delta, double gamma,
                   double* out);

/* Prox of the I-divergence data term, Eq. subproblemGIdiv, per element. */
double orc_prox(double ut, double f, double lam);
void orc_prox_vec(const double* ut, const double* f, long n, double lam, double* u);
/* du/du~ (Eq. derv2) and du/dlam (Eq. derv4) per element. */
double orc_prox_du(double ut, double f, double lam);
double orc_prox_dlam(double ut, double f, double lam);

/* Data terms of a stage (the reaction force):
 *   ORC_IDIV  0: despeckling, u_t = prox of G = lam <u^2 - 2 f^2 log u, 1>
 *                at u~ = u_{t-1} - diffusion (Eqs. diffusionprocessfinal,
 *                subproblemGIdiv);
 *   ORC_GAUSS 1: TNRD Gaussian denoising, G = 0, D = lam/2 |u - f|^2 (Sec. 2.2.1,
 *                A = identity): u_t = u_{t-1} - diffusion - lam (u_{t-1} - f);
 *   ORC_PROJ  2: the explicit despeckling step with projection, Eq.
 *                diffusion_backP: u~ = u_{t-1} - diffusion
 *                - (lam / u_{t-1}) (1 - f^2 / u_{t-1}^2), u_t = max(u~, c). */
enum { ORC_IDIV = 0, ORC_GAUSS = 1, ORC_PROJ = 2 };

/* One stage t (0-based) of the model with data term `mode` (c: the projection
 * floor of ORC_PROJ, unused otherwise).  ut_out (nullable) receives u~. */
void orc_stage_mode(const double* u_prev, const double* f, int H, int W, int t,
                    const double* k, const double* w, const double* lam,
                    int nk, int ks, int nrbf, double mu0, double delta, double gamma,
                    int mode, double c, double* u_next, double* ut_out);
void orc_forward_mode(const double* f, int H, int W, int T,
                      const double* k, const double* w, const double* lam,
                      int nk, int ks, int nrbf, double mu0, double delta, double gamma,
                      int mode, double c, double* u_all);
void orc_backward_mode(const double* f, int H, int W, int T,
                       const double* k, const double* w, const double* lam,
                       int nk, int ks, int nrbf, double mu0, double delta, double gamma,
                       int mode, double c, const double* u_all, const double* e_T,
                       double* e_0, double* gk, double* gw, double* glam);

/* One stage t (0-based) of the model: u_next = prox(u_prev - diffusion).
 * ut_out (nullable) receives u~.  (orc_stage_mode with ORC_IDIV.) */
void orc_stage(const double* u_prev, const double* f, int H, int W, int t,
               const double* k, const double* w, const double* lam,
               int nk, int ks, int nrbf, double mu0, double delta, double gamma,
               double* u_next, double* ut_out);

/* T stages from u_0 = f; u_all receives u_0..u_T, [T+1][H][W].  (ORC_IDIV.) */
void orc_forward(const double* f, int H, int W, int T,
                 const double* k, const double* w, const double* lam,
                 int nk, int ks, int nrbf, double mu0, double delta, double gamma,
                 double* u_all);

/* Gradients of a loss L given e_T = dL/du_T (one image), by Eq. iterstep.
 * Outputs are overwritten: e_0 = dL/du_0 [H][W] (nullable), gk [T][nk][ks][ks],
 * gw [T][nk][nrbf], glam [T].  Requires lam_t > 0.  (ORC_IDIV.) */
void orc_backward(const double* f, int H, int W, int T,
                  const double* k, const double* w, const double* lam,
                  int nk, int ks, int nrbf, double mu0, double delta, double gamma,
                  const double* u_all, const double* e_T,
                  double* e_0, double* gk, double* gw, double* glam);

/* OpenMP thread control (1 when built without OpenMP). */
void orc_set_threads(int n);
int orc_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif
