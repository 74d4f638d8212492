/*
 * FP64 CPU oracle for the Monte-Carlo ELBO step of variational sparse Bayesian
 * crystalline-phase search (Murakami et al., arXiv 2501.09308).
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the package smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header,
 * table or constant generator with the CUDA path; the only common input is the
 * seeded synthetic data.
 *
 * It is deliberately plain: every quantity is computed in double precision by
 * the direct loops of the paper's definitions, with no blocking, windowing or
 * reordering.  Each function names the passage it follows.  Readings of points
 * the paper leaves open are marked "Reading:" and are the same readings the
 * CUDA path takes.
 *
 * Parameter layout.  Per phase k the five physical parameters are, in this
 * order, j = 0 intensity h_k, 1 peak shift mu_k, 2 width w_k (FWHM, degrees),
 * 3 Gauss-Lorentz ratio r_k, 4 asymmetry alpha_k (Appendix A.2, Appendix B.2).
 * The variational family is a mean-field Gaussian (Sec. 3.2, the product of
 * normals) over the unconstrained u_kj, with u = loc + softplus(raw) * eps and
 *   h = exp(u0), mu = u1, w = exp(u2), r = sigmoid(u3), alpha = u4.
 * (Reading: the paper states q as normal over each parameter but h, w > 0 and
 * r in [0, 1]; the normal is placed on the log / logit scale for those.)
 * Gradient layout: grad[k*10 + j] = dELBO/dloc[k][j], grad[k*10 + 5 + j] =
 * dELBO/draw[k][j].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_LN2 0.69314718055994530942
#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11). */
/* Ten rounds of: two 32x32->64 multiplies by the fixed multipliers, the high */
/* halves xored with the other two words and the round key, then a key bump  */
/* by the two Weyl increments.                                               */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in (0,1) from the top 24 bits, exactly representable in f32/f64. */
static double orc_u01(uint32_t v) { return ((double)(v >> 8) + 0.5) * (1.0 / 16777216.0); }

/*
 * Standard normals for the reparameterised draw (Sec. 3.2; Reading: Box-Muller
 * on Philox output).  For sample s, phase k, step iter and stream tag, the
 * counter is (s, k, iter, tag*256 + j) for j = 0, 1 and the key is the 64-bit
 * seed.  The eight uniforms u0..u7 form Box-Muller pairs (u0,u1), (u2,u3), ...
 * giving z_{2q} = sqrt(-2 ln u_{2q}) cos(2 pi u_{2q+1}) and z_{2q+1} the sine;
 * the first five are eps[s][k][0..4].
 */
void orc_normals(uint64_t seed, uint32_t tag, uint32_t iter, int S, int K, double *eps)
{
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    for (int s = 0; s < S; ++s) {
        for (int k = 0; k < K; ++k) {
            double z[8];
            for (int j = 0; j < 2; ++j) {
                uint32_t ctr[4] = {(uint32_t)s, (uint32_t)k, iter, tag * 256u + (uint32_t)j};
                uint32_t o[4];
                orc_philox4x32_10(ctr, key, o);
                for (int q = 0; q < 2; ++q) {
                    double u1 = orc_u01(o[2 * q]), u2 = orc_u01(o[2 * q + 1]);
                    double rad = sqrt(-2.0 * log(u1));
                    z[4 * j + 2 * q] = rad * cos(2.0 * ORC_PI * u2);
                    z[4 * j + 2 * q + 1] = rad * sin(2.0 * ORC_PI * u2);
                }
            }
            for (int j = 0; j < 5; ++j) eps[((size_t)s * K + k) * 5 + j] = z[j];
        }
    }
}

double orc_softplus(double x);
double orc_sigmoid(double x);

/*
 * Logistic noise of the gate variant: for sample s, phase k, step iter and
 * stream tag, the first output of Philox4x32-10 at counter
 * (s, k, iter, tag*256 + 2) gives u in (0, 1) and L = ln u - ln(1 - u).
 */
void orc_gate_noise(uint64_t seed, uint32_t tag, uint32_t iter, int S, int K, double *L)
{
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    for (int s = 0; s < S; ++s)
        for (int k = 0; k < K; ++k) {
            uint32_t c[4] = {(uint32_t)s, (uint32_t)k, iter, tag * 256u + 2u}, o[4];
            orc_philox4x32_10(c, key, o);
            double u = orc_u01(o[0]);
            L[(size_t)s * K + k] = log(u) - log1p(-u);
        }
}

/*
 * Binary-Concrete gate (Maddison, Mnih & Teh, "The Concrete Distribution",
 * ICLR 2017; Reading: a model variant, not in the paper, whose sparsity comes
 * from the exponential prior on h).  With location a (a logit), temperature
 * tau and logistic noise L, y = (a + L) / tau and the gate is z = sigmoid(y).
 * The density of y is
 *   ln q(y) = ln tau + a - tau y - 2 softplus(a - tau y),
 * and the prior is the same family with location a0 = ln(pi0/(1 - pi0)) and
 * the same temperature.  Per draw and phase the objective gains
 * ln p(y) - ln q(y); its reparameterisation gradient in a is
 * (1/tau) [dLL/dy + d ln p/dy] (the ln q terms cancel for a location family),
 * with d ln p/dy = tau (2 sigmoid(a0 - tau y) - 1) and dLL/dy = dLL/dz z(1-z).
 * Writes z and returns ln p(y) - ln q(y); *dlnp_dy receives d ln p/dy.
 */
double orc_gate_terms(double a, double L, double tau, double a0, double *z, double *dlnp_dy)
{
    double y = (a + L) / tau;
    *z = orc_sigmoid(y);
    double lq = log(tau) + a - tau * y - 2.0 * orc_softplus(a - tau * y);
    double lp = log(tau) + a0 - tau * y - 2.0 * orc_softplus(a0 - tau * y);
    *dlnp_dy = tau * (2.0 * orc_sigmoid(a0 - tau * y) - 1.0);
    return lp - lq;
}

/* ------------------------------------------------------------------------ */
/* Variational transform                                                    */
/* ------------------------------------------------------------------------ */
double orc_softplus(double x) { return x > 0 ? x + log1p(exp(-x)) : log1p(exp(x)); }
double orc_sigmoid(double x) { return x >= 0 ? 1.0 / (1.0 + exp(-x)) : exp(x) / (1.0 + exp(x)); }

/* u = loc + softplus(raw) * eps and theta = (e^u0, u1, e^u2, sigmoid(u3), u4). */
void orc_theta(int S, int K, const double *loc, const double *raw, const double *eps,
               double *u, double *theta)
{
    for (int s = 0; s < S; ++s)
        for (int k = 0; k < K; ++k)
            for (int j = 0; j < 5; ++j) {
                size_t i = ((size_t)s * K + k) * 5 + j;
                double uj = loc[k * 5 + j] + orc_softplus(raw[k * 5 + j]) * eps[i];
                u[i] = uj;
                double th;
                switch (j) {
                case 0: th = exp(uj); break;
                case 1: th = uj; break;
                case 2: th = exp(uj); break;
                case 3: th = orc_sigmoid(uj); break;
                default: th = uj; break;
                }
                theta[i] = th;
            }
}

/* ------------------------------------------------------------------------ */
/* Profile function (Appendix A.2)                                           */
/* ------------------------------------------------------------------------ */
/*
 * Gaussian and Lorentzian components at offset d = x - rho with FWHM w and
 * asymmetry alpha (already clamped).  Reading: G and L are height-normalised
 * with full width at half maximum equal to the side width; the asymmetry
 * function A multiplies the width on the x >= rho side (so the peak stays
 * continuous at rho), the x < rho side keeps w.
 *   t = d / (A w),  G = exp(-4 ln2 t^2),  L = 1 / (1 + 4 t^2).
 */
void orc_components(double d, double w, double alpha_c, double *G, double *L)
{
    double side = d >= 0.0 ? alpha_c * w : w;
    double t = d / side;
    *G = exp(-4.0 * ORC_LN2 * t * t);
    *L = 1.0 / (1.0 + 4.0 * t * t);
}

/* Width factor of the angle-dependent variant at 2-theta x (degrees):
 * sec(theta) with theta = x / 2, i.e. 1 / cos(x pi / 360). */
double orc_sec(double x) { return 1.0 / cos(x * ORC_PI / 360.0); }

/*
 * Area of the height-normalised split pseudo-Voigt of unit height (the
 * closed form of the area-ratio reading, Sec. 4): the Gaussian and Lorentzian
 * halves of FWHM w on the left and alpha w on the right integrate to
 *   a(w, alpha, r) = ((1 + alpha) w / 2) [(1 - r) sqrt(pi / ln 2) / 2 + r pi / 2].
 * The area-normalised variant divides each phase's profile by it.
 */
double orc_area_factor(double w, double alpha_c, double r)
{
    return 0.5 * (1.0 + alpha_c) * w * ((1.0 - r) * 0.5 * sqrt(ORC_PI / ORC_LN2) + r * 0.5 * ORC_PI);
}

/* Pseudo-Voigt V = (1 - r) G + r L (Appendix A.2, profile of one peak). */
double orc_pvoigt(double d, double w, double r, double alpha_c)
{
    double G, L;
    orc_components(d, w, alpha_c, &G, &L);
    return (1.0 - r) * G + r * L;
}

/*
 * f(x_i) = B(x_i) + sum_k h_k sum_m I_m V(x_i; p_m + mu_k, w_k, r_k, alpha_k),
 * the signal of the eq. labelled "signal" plus the fixed background, by the
 * direct triple loop over phases, peaks and points (Sec. 2.3).  theta is
 * [S][K][5]; f is [S][N].  alpha is clamped below at alpha_min (Reading: the
 * normal q and prior on alpha admit alpha <= 0, where the profile is undefined).
 */
void orc_profile_ex(int K, const int *off, const double *pos, const double *inten,
                    int N, const double *x, const double *bg,
                    int S, const double *theta, double alpha_min, int sec, int area_norm, double *f)
{
#pragma omp parallel for schedule(dynamic)
    for (int s = 0; s < S; ++s) {
        for (int i = 0; i < N; ++i) {
            double acc = bg[i];
            for (int k = 0; k < K; ++k) {
                const double *th = theta + ((size_t)s * K + k) * 5;
                double h = th[0], mu = th[1], w = th[2], r = th[3];
                double ac = th[4] > alpha_min ? th[4] : alpha_min;
                double C = 0.0, wx = sec ? w * orc_sec(x[i]) : w;
                for (int m = off[k]; m < off[k + 1]; ++m) {
                    double d = x[i] - (pos[m] + mu);
                    C += inten[m] * orc_pvoigt(d, wx, r, ac);
                }
                if (area_norm) C /= orc_area_factor(w, ac, r);
                acc += h * C;
            }
            f[(size_t)s * N + i] = acc;
        }
    }
}

void orc_profile(int K, const int *off, const double *pos, const double *inten,
                 int N, const double *x, const double *bg,
                 int S, const double *theta, double alpha_min, double *f)
{
    orc_profile_ex(K, off, pos, inten, N, x, bg, S, theta, alpha_min, 0, 0, f);
}

/*
 * Background variant (Reading: the paper fixes B beforehand, App. A.2; here a
 * smooth multiplicative correction is fitted with the phases):
 *   B_i(beta) = B_i exp(beta_0 T_0(z_i) + beta_1 T_1(z_i) + beta_2 T_2(z_i)),
 * T_0 = 1, T_1 = z, T_2 = 2 z^2 - 1 (Chebyshev), z_i = 2 (x_i - x_0) /
 * (x_{N-1} - x_0) - 1 in [-1, 1] (z = 0 when N = 1).  Each beta_j has the
 * prior N(0, bg_sd^2) and is point-estimated (its q is a point mass): the
 * objective adds ln p(beta) to every draw's log joint.
 * Writes Bb[N] = B_i(beta) and T[3*N] = T_j(z_i).
 */
void orc_background(int N, const double *x, const double *bg, const double *beta, double *Bb, double *T)
{
    for (int i = 0; i < N; ++i) {
        double z = N > 1 ? 2.0 * (x[i] - x[0]) / (x[N - 1] - x[0]) - 1.0 : 0.0;
        double t0 = 1.0, t1 = z, t2 = 2.0 * z * z - 1.0;
        if (T) { T[i] = t0; T[N + i] = t1; T[2 * N + i] = t2; }
        Bb[i] = bg[i] * exp(beta[0] * t0 + beta[1] * t1 + beta[2] * t2);
    }
}

/* ln p(beta) = sum_j ln N(beta_j; 0, bg_sd^2). */
double orc_background_prior(const double *beta, double bg_sd)
{
    double s = 0.0;
    for (int j = 0; j < 3; ++j) s += -0.5 * (beta[j] / bg_sd) * (beta[j] / bg_sd) - log(bg_sd) - 0.5 * log(2.0 * ORC_PI);
    return s;
}

/* ------------------------------------------------------------------------ */
/* Poisson likelihood (Appendix A.2)                                         */
/* ------------------------------------------------------------------------ */
/* ln p(Y|Phi) = sum_i [ y_i ln f_i - f_i - ln y_i! ]  (direct form). */
double orc_loglik_direct(int N, const double *y, const double *f)
{
    double ll = 0.0;
    for (int i = 0; i < N; ++i) {
        double yl = y[i] > 0.0 ? y[i] * log(f[i]) : 0.0;
        ll += yl - f[i] - lgamma(y[i] + 1.0);
    }
    return ll;
}

/*
 * The same sum split into a data constant c_i = y ln y - y - ln y! and the
 * deviance part D_i = y ln(f/y) - (f - y) (D_i = -f when y = 0).  Exactly
 * equal to the direct form in real arithmetic.
 */
double orc_loglik_deviance(int N, const double *y, const double *f, double *csum_out)
{
    double c = 0.0, dsum = 0.0;
    for (int i = 0; i < N; ++i) {
        if (y[i] > 0.0) {
            c += y[i] * log(y[i]) - y[i] - lgamma(y[i] + 1.0);
            dsum += y[i] * log(f[i] / y[i]) - (f[i] - y[i]);
        } else {
            dsum += -f[i];
        }
    }
    if (csum_out) *csum_out = c;
    return c + dsum;
}

/*
 * Likelihood variant: Gaussian with variance v_i = max(y_i, 1), a weighted
 * residual sum of squares (not the paper's model, which is Poisson,
 * Appendix A.2; v_i is the Poisson variance where counts are large):
 *   ln p(Y|Phi) = sum_i [ -(y_i - f_i)^2 / (2 v_i) - ln(2 pi v_i) / 2 ],
 * with d/df_i = (y_i - f_i) / v_i.
 */
double orc_gauss_var(double y) { return y > 1.0 ? y : 1.0; }

double orc_loglik_gauss(int N, const double *y, const double *f)
{
    double s = 0.0;
    for (int i = 0; i < N; ++i) {
        double v = orc_gauss_var(y[i]), r = y[i] - f[i];
        s += -0.5 * r * r / v - 0.5 * log(2.0 * ORC_PI * v);
    }
    return s;
}

/* ------------------------------------------------------------------------ */
/* Priors (Sec. 2.2, Appendix B.2) and the log-Jacobian of the transform     */
/* ------------------------------------------------------------------------ */
typedef struct {
    double lambda;      /* rate of the exponential prior on h: 1 / max(Y - B)   */
    double mu_sd;       /* mu ~ Norm(0, mu_sd)                                  */
    double alpha_mean;  /* alpha ~ Norm(alpha_mean, alpha_sd)                   */
    double alpha_sd;
    double w_shape;     /* w ~ Gam(shape, rate)   (Reading: rate, mean 0.03 deg) */
    double w_rate;
    double alpha_min;   /* profile clamp on alpha                               */
} orc_prior;

/*
 * Model and estimator variants (none is the paper's model; all zero gives it):
 *   lik     0 Poisson, 1 Gaussian with variance max(y, 1)   (orc_loglik_gauss)
 *   iw      0 ELBO, 1 importance-weighted bound              (orc_iw_weights)
 *   shared  1: one shape draw per step for all samples       (orc_tie_shapes)
 *   sec     1: angle-dependent width, every side width at point x multiplied
 *           by sec(theta), theta = x / 2 (x = 2-theta in degrees)   (orc_sec)
 *   bgfit   1: background fitted in-model                   (orc_background)
 *   gates   1: explicit phase gates z = sigmoid((a + L)/tau) scale each
 *           phase's profile (not in the paper; orc_gate_terms)
 *   area_norm 1: each phase's profile divided by its area per unit height
 *           (orc_area_factor), so h is an integrated intensity
 *   fix_r, fix_alpha  1: r / alpha held at a given value: a constant of the
 *           model, not a parameter of q (no prior, Jacobian, entropy, ln q
 *           or gradient term; orc_fixed_terms)
 */
typedef struct {
    int lik, iw, shared, sec;
    int bgfit;            /* 1: fitted background correction (orc_background)      */
    double bg_sd;         /* prior standard deviation of each coefficient beta_j  */
    double *beta;         /* [3] coefficients (in; orc_fit_ex updates them)        */
    double *grad_beta;    /* [3] d objective / d beta (orc_elbo_grad_ex; may be NULL) */
    double *m_beta, *v_beta;   /* [3] their Adam moments (orc_fit_ex)              */
    int fix_r, fix_alpha;      /* 1: r / alpha held at r_value / alpha_value       */
    double r_value, alpha_value;
    int area_norm;             /* 1: area-normalised profiles (orc_area_factor)    */
    int gates;                 /* 1: binary-Concrete phase gates (orc_gate_terms)   */
    double gate_tau, gate_prior_logit;   /* temperature; prior logit ln(pi0 / (1 - pi0)) */
    double *gate_a;            /* [K] gate logits (in; orc_fit_ex updates them)     */
    double *grad_gate;         /* [K] d objective / d gate_a (may be NULL)          */
    double *m_gate, *v_gate;   /* [K] their Adam moments (orc_fit_ex)               */
    const double *gate_noise;  /* [S*K] logistic noise L (orc_gate_noise)           */
} orc_variant;

/* ln p(theta) for one phase: Exp(lambda) on h, normal on mu and alpha,
   Uni(0,1) on r (log density 0), gamma on w. */
double orc_log_prior(const orc_prior *pr, const double *th)
{
    double h = th[0], mu = th[1], w = th[2], al = th[4];
    double lp = log(pr->lambda) - pr->lambda * h;
    lp += -0.5 * (mu / pr->mu_sd) * (mu / pr->mu_sd) - log(pr->mu_sd) - 0.5 * log(2.0 * ORC_PI);
    double za = (al - pr->alpha_mean) / pr->alpha_sd;
    lp += -0.5 * za * za - log(pr->alpha_sd) - 0.5 * log(2.0 * ORC_PI);
    lp += pr->w_shape * log(pr->w_rate) - lgamma(pr->w_shape) + (pr->w_shape - 1.0) * log(w) - pr->w_rate * w;
    return lp;
}

/* ln |d theta / d u| = u_h + u_w + ln r + ln(1 - r). */
double orc_log_jac(const double *u)
{
    return u[0] + u[2] - orc_softplus(-u[3]) - orc_softplus(u[3]);
}

/* d/du [ln p(theta(u)) + ln|J|] per parameter. */
static void orc_prior_jac_grad(const orc_prior *pr, const double *th, double *g)
{
    g[0] = 1.0 - pr->lambda * th[0];
    g[1] = -th[1] / (pr->mu_sd * pr->mu_sd);
    g[2] = pr->w_shape - pr->w_rate * th[2];
    g[3] = 1.0 - 2.0 * th[3];
    g[4] = -(th[4] - pr->alpha_mean) / (pr->alpha_sd * pr->alpha_sd);
}

/* Entropy of the mean-field normal: sum_kj [ln sigma_kj + (1 + ln 2 pi) / 2]. */
double orc_entropy(int K, const double *raw)
{
    double H = 0.0;
    for (int i = 0; i < 5 * K; ++i) H += log(orc_softplus(raw[i])) + 0.5 * (1.0 + log(2.0 * ORC_PI));
    return H;
}

/*
 * Parameters held fixed (orc_variant.fix_r / fix_alpha) leave q: per draw
 * the ln p + ln|J| terms of a fixed r (its Jacobian ln r(1-r); the uniform
 * prior adds nothing) and of a fixed alpha (its normal prior) are removed,
 * and so are their entropy and ln q terms.  Returns the ln p + ln|J| part
 * to subtract for one phase of one draw (u, theta of that phase).
 */
double orc_fixed_lpj(const orc_prior *pr, const orc_variant *var, const double *u, const double *th)
{
    double d = 0.0;
    if (var && var->fix_r) d += -orc_softplus(-u[3]) - orc_softplus(u[3]);
    if (var && var->fix_alpha) {
        double za = (th[4] - pr->alpha_mean) / pr->alpha_sd;
        d += -0.5 * za * za - log(pr->alpha_sd) - 0.5 * log(2.0 * ORC_PI);
    }
    return d;
}

/* Is parameter j of q free (not held fixed)? */
int orc_free(const orc_variant *var, int j)
{
    return !(var && ((j == 3 && var->fix_r) || (j == 4 && var->fix_alpha)));
}

/* ------------------------------------------------------------------------ */
/* Importance-weighted bound (estimator variant)                              */
/* ------------------------------------------------------------------------ */
/*
 * The importance-weighted bound of Burda, Grosse & Salakhutdinov
 * ("Importance Weighted Autoencoders", ICLR 2016) on the S draws of one step:
 *   L_S = ln (1/S) sum_s w_s,
 *   ln w_s = ln p(Y|theta_s) + ln p(theta_s) + ln|J_s| - ln q(u_s),
 *   ln q(u_s) = sum_kj [ -eps_skj^2 / 2 - ln sigma_kj - ln(2 pi) / 2 ].
 * L_1 is the single-draw ELBO with the entropy replaced by -ln q(u_1), and
 * L_S >= mean_s ln w_s.  With wt_s = w_s / sum_s' w_s' and G_s as for the
 * ELBO, its reparameterisation gradient (eps fixed) is
 *   dL_S/dloc = sum_s wt_s G_s,
 *   dL_S/draw = [ sum_s wt_s G_s eps_s + 1/sigma ] sigmoid(raw),
 * the 1/sigma being the derivative of -ln q(u_s) with u_s = loc + sigma eps_s.
 * Returns L_S and writes wt[S]; ll and lpj are the per-draw terms; parameters
 * held fixed by var are not part of q.
 */
double orc_iw_weights(int K, int S, const double *raw, const double *eps, const double *ll,
                      const double *lpj, const orc_variant *var, double *wt)
{
    double *lw = (double *)malloc((size_t)S * sizeof(double));
    double mx = -INFINITY;
    for (int s = 0; s < S; ++s) {
        double lq = 0.0;
        for (int i = 0; i < 5 * K; ++i) {
            if (!orc_free(var, i % 5)) continue;   /* held fixed: not part of q */
            double e = eps[(size_t)s * K * 5 + i];
            lq += -0.5 * e * e - log(orc_softplus(raw[i])) - 0.5 * log(2.0 * ORC_PI);
        }
        lw[s] = ll[s] + lpj[s] - lq;
        if (lw[s] > mx) mx = lw[s];
    }
    double sum = 0.0;
    for (int s = 0; s < S; ++s) sum += exp(lw[s] - mx);
    for (int s = 0; s < S; ++s) wt[s] = exp(lw[s] - mx) / sum;
    free(lw);
    return mx + log(sum) - log((double)S);
}

/* ------------------------------------------------------------------------ */
/* Monte-Carlo ELBO and its gradient (Sec. 3.2)                               */
/* ------------------------------------------------------------------------ */
/*
 * ELBO estimate  L = (1/S) sum_s [ln p(Y|theta_s) + ln p(theta_s) + ln|J_s|] + H(q)
 * with theta_s = theta(loc + sigma * eps_s), and its exact gradient with
 * respect to loc and raw (the reparameterisation gradient of this estimator).
 *
 * Likelihood gradient: with g_i = y_i / f_i - 1,
 *   dLL/dh_k     = sum_i g_i C_k(x_i)
 *   dLL/dmu_k    = h_k sum_i g_i sum_m I_m dV/dmu
 *   dLL/dw_k, dLL/dalpha_k, dLL/dr_k likewise (alpha only on the d >= 0 side,
 *   and zero while alpha is held at the clamp).
 * Chain to u: dtheta/du = (h, 1, w, r(1-r), 1).  Then
 *   dL/dloc = mean_s G_s,  dL/draw = [mean_s G_s eps_s + 1/sigma] sigmoid(raw).
 *
 * Outputs: elbo; ll[S], lpj[S] (log prior + log Jacobian) if non-NULL;
 * grad[K*10] if non-NULL; f[S*N] if non-NULL.
 *
 * orc_elbo_grad_ex also takes the variants (orc_variant; NULL = none): the
 * likelihood (lik: the Gaussian's g_i = (y_i - f_i)/v_i replaces
 * y_i/f_i - 1), the objective (iw: the importance weights replace the 1/S of
 * the sample means; `elbo` then receives that objective) and the
 * angle-dependent width (sec: every side width at point x_i is multiplied by
 * sec(x_i / 2), so t = d / side keeps its form and so do dt/dw = -t/w and
 * dt/dalpha = -t/alpha, while dt/dmu = -1/side carries the factor).
 */
void orc_elbo_grad_ex(int K, const int *off, const double *pos, const double *inten,
                      int N, const double *x, const double *y, const double *bg,
                      const orc_prior *pr, const orc_variant *var, int S, const double *loc, const double *raw,
                      const double *eps, double *elbo, double *ll, double *lpj,
                      double *grad, double *f_out)
{
    const int lik = var ? var->lik : 0, iw = var ? var->iw : 0, sec = var ? var->sec : 0;
    const int bgfit = var ? var->bgfit : 0;
    const int gates = var ? var->gates : 0;
    double *gg = gates ? (double *)calloc((size_t)S * K, sizeof(double)) : NULL;   /* per-draw gate gradients */
    double *Bb = NULL, *Tb = NULL, *gbs = NULL, lpb = 0.0;
    if (bgfit) {   /* fitted background: B(beta), its Chebyshev terms, per-draw beta sums */
        Bb = (double *)malloc((size_t)N * sizeof(double));
        Tb = (double *)malloc((size_t)3 * N * sizeof(double));
        gbs = (double *)calloc((size_t)S * 3, sizeof(double));
        orc_background(N, x, bg, var->beta, Bb, Tb);
        lpb = orc_background_prior(var->beta, var->bg_sd);
        bg = Bb;
    }
    size_t SK5 = (size_t)S * K * 5;
    double *u = (double *)malloc(SK5 * sizeof(double));
    double *th = (double *)malloc(SK5 * sizeof(double));
    double *G = (double *)calloc(SK5, sizeof(double));
    double *lls = (double *)malloc((size_t)S * sizeof(double));
    double *lps = (double *)malloc((size_t)S * sizeof(double));
    orc_theta(S, K, loc, raw, eps, u, th);
    if (var && (var->fix_r || var->fix_alpha))   /* fixed r / alpha: model constants */
        for (size_t i = 0; i < (size_t)S * K; ++i) {
            if (var->fix_r) th[i * 5 + 3] = var->r_value;
            if (var->fix_alpha) th[i * 5 + 4] = var->alpha_value;
        }

#pragma omp parallel for schedule(dynamic)
    for (int s = 0; s < S; ++s) {
        double *f = (double *)malloc((size_t)N * sizeof(double));
        double *gi = (double *)malloc((size_t)N * sizeof(double));
        const double *ths = th + (size_t)s * K * 5;
        const double *us = u + (size_t)s * K * 5;
        /* gates: z_k of this draw, its ln p - ln q and d ln p / dy */
        double *zg = NULL, *dpg = NULL, glp = 0.0;
        if (gates) {
            zg = (double *)malloc((size_t)K * sizeof(double));
            dpg = (double *)malloc((size_t)K * sizeof(double));
            for (int k = 0; k < K; ++k)
                glp += orc_gate_terms(var->gate_a[k], var->gate_noise[(size_t)s * K + k], var->gate_tau,
                                      var->gate_prior_logit, &zg[k], &dpg[k]);
        }
        /* forward: profile, likelihood */
        for (int i = 0; i < N; ++i) {
            double acc = bg[i];
            for (int k = 0; k < K; ++k) {
                const double *t = ths + k * 5;
                double ac = t[4] > pr->alpha_min ? t[4] : pr->alpha_min;
                double C = 0.0;
                double wx = sec ? t[2] * orc_sec(x[i]) : t[2];   /* width at this point */
                for (int m = off[k]; m < off[k + 1]; ++m)
                    C += inten[m] * orc_pvoigt(x[i] - (pos[m] + t[1]), wx, t[3], ac);
                if (var && var->area_norm) C /= orc_area_factor(t[2], ac, t[3]);
                acc += t[0] * C * (gates ? zg[k] : 1.0);
            }
            f[i] = acc;
            gi[i] = lik ? (y[i] - acc) / orc_gauss_var(y[i]) : y[i] / acc - 1.0;
        }
        if (f_out) memcpy(f_out + (size_t)s * N, f, (size_t)N * sizeof(double));
        lls[s] = lik ? orc_loglik_gauss(N, y, f) : orc_loglik_direct(N, y, f);
        double lp = lpb + glp;   /* ln p(beta) of the fitted background, gate terms (0 otherwise) */
        for (int k = 0; k < K; ++k)
            lp += orc_log_prior(pr, ths + k * 5) + orc_log_jac(us + k * 5) - orc_fixed_lpj(pr, var, us + k * 5, ths + k * 5);
        lps[s] = lp;
        if (bgfit)   /* d LL_s / d beta_j = sum_i g_i B_i(beta) T_j(z_i) */
            for (int j = 0; j < 3; ++j)
                for (int i = 0; i < N; ++i) gbs[(size_t)s * 3 + j] += gi[i] * Bb[i] * Tb[(size_t)j * N + i];
        /* backward: per-phase likelihood gradient in theta, chained to u */
        for (int k = 0; k < K; ++k) {
            const double *t = ths + k * 5;
            double h0 = t[0], mu = t[1], w = t[2], r = t[3], al = t[4];
            double h = gates ? h0 * zg[k] : h0;   /* the phase's profile scale */
            int clamped = !(al > pr->alpha_min);
            double ac = clamped ? pr->alpha_min : al;
            double dh = 0, dmu = 0, dw = 0, dr = 0, dal = 0;
            for (int i = 0; i < N; ++i) {
                double C = 0, Cmu = 0, Cw = 0, Cr = 0, Cal = 0;
                for (int m = off[k]; m < off[k + 1]; ++m) {
                    double d = x[i] - (pos[m] + mu);
                    double side = (d >= 0.0 ? ac * w : w) * (sec ? orc_sec(x[i]) : 1.0);
                    double tt = d / side;
                    double Gc = exp(-4.0 * ORC_LN2 * tt * tt);
                    double Lc = 1.0 / (1.0 + 4.0 * tt * tt);
                    double V = (1.0 - r) * Gc + r * Lc;
                    /* dV/dt for t = d / side */
                    double dVdt = (1.0 - r) * (-8.0 * ORC_LN2 * tt * Gc) + r * (-8.0 * tt * Lc * Lc);
                    double I = inten[m];
                    C += I * V;
                    Cmu += I * dVdt * (-1.0 / side);          /* d t / d mu = -1 / side   */
                    Cw += I * dVdt * (-tt / w);               /* d t / d w  = -t / w      */
                    Cr += I * (Lc - Gc);                      /* d V / d r  = L - G        */
                    if (d >= 0.0 && !clamped) Cal += I * dVdt * (-tt / ac); /* d t / d alpha */
                }
                if (var && var->area_norm) {
                    /* f = h C / a(w, alpha, r): product rule with d ln a / dw = 1/w,
                       d ln a / d alpha = 1/(1 + alpha), d ln a / dr as below */
                    double a = orc_area_factor(w, ac, r);
                    double A = (1.0 - r) * 0.5 * sqrt(ORC_PI / ORC_LN2) + r * 0.5 * ORC_PI;
                    double dlna_dr = (0.5 * ORC_PI - 0.5 * sqrt(ORC_PI / ORC_LN2)) / A;
                    dh += gi[i] * C / a;
                    dmu += gi[i] * h * Cmu / a;
                    dw += gi[i] * h * (Cw - C / w) / a;
                    dr += gi[i] * h * (Cr - C * dlna_dr) / a;
                    if (!clamped) dal += gi[i] * h * (Cal - C / (1.0 + ac)) / a;
                    continue;
                }
                dh += gi[i] * C;
                dmu += gi[i] * h * Cmu;
                dw += gi[i] * h * Cw;
                dr += gi[i] * h * Cr;
                dal += gi[i] * h * Cal;
            }
            double pj[5];
            orc_prior_jac_grad(pr, t, pj);
            double *Gs = G + ((size_t)s * K + k) * 5;
            Gs[0] = dh * h + pj[0];
            if (gates)   /* dLL/dz = h0 dh; dy: times z(1 - z); then (1/tau)(dLL/dy + d ln p/dy) */
                gg[(size_t)s * K + k] = (h0 * dh * zg[k] * (1.0 - zg[k]) + dpg[k]) / var->gate_tau;
            Gs[1] = dmu + pj[1];
            Gs[2] = dw * w + pj[2];
            Gs[3] = orc_free(var, 3) ? dr * r * (1.0 - r) + pj[3] : 0.0;
            Gs[4] = orc_free(var, 4) ? dal + pj[4] : 0.0;
        }
        free(f);
        free(gi);
        free(zg);
        free(dpg);
    }

    /* sample weights: 1/S for the ELBO; for the importance-weighted bound the
       normalised weights w_s / sum w (Burda et al.), see orc_iw_weights */
    double *wt = (double *)malloc((size_t)S * sizeof(double));
    if (iw) {
        *elbo = orc_iw_weights(K, S, raw, eps, lls, lps, var, wt);
    } else {
        double acc = 0.0;
        for (int s = 0; s < S; ++s) acc += lls[s] + lps[s];
        double H = orc_entropy(K, raw);
        for (int k = 0; k < K; ++k)   /* fixed parameters carry no entropy */
            for (int j = 3; j < 5; ++j)
                if (!orc_free(var, j)) H -= log(orc_softplus(raw[k * 5 + j])) + 0.5 * (1.0 + log(2.0 * ORC_PI));
        *elbo = acc / S + H;
        for (int s = 0; s < S; ++s) wt[s] = 1.0 / S;
    }
    if (ll) memcpy(ll, lls, (size_t)S * sizeof(double));
    if (lpj) memcpy(lpj, lps, (size_t)S * sizeof(double));
    if (grad) {
        for (int k = 0; k < K; ++k)
            for (int j = 0; j < 5; ++j) {
                double gl = 0.0, ge = 0.0;
                for (int s = 0; s < S; ++s) {
                    size_t i = ((size_t)s * K + k) * 5 + j;
                    gl += wt[s] * G[i];
                    ge += wt[s] * G[i] * eps[i];
                }
                double rw = raw[k * 5 + j];
                grad[k * 10 + j] = gl;
                grad[k * 10 + 5 + j] = orc_free(var, j) ? (ge + 1.0 / orc_softplus(rw)) * orc_sigmoid(rw) : 0.0;
            }
    }
    if (gates && var->grad_gate)
        for (int k = 0; k < K; ++k) {
            double gsum = 0.0;
            for (int s = 0; s < S; ++s) gsum += wt[s] * gg[(size_t)s * K + k];
            var->grad_gate[k] = gsum;
        }
    free(gg);
    if (bgfit && var->grad_beta)
        for (int j = 0; j < 3; ++j) {
            double gsum = 0.0;
            for (int s = 0; s < S; ++s) gsum += wt[s] * gbs[(size_t)s * 3 + j];
            var->grad_beta[j] = gsum - var->beta[j] / (var->bg_sd * var->bg_sd);
        }
    free(u); free(th); free(G); free(lls); free(lps); free(wt);
    free(Bb); free(Tb); free(gbs);
}

void orc_elbo_grad(int K, const int *off, const double *pos, const double *inten,
                   int N, const double *x, const double *y, const double *bg,
                   const orc_prior *pr, int S, const double *loc, const double *raw,
                   const double *eps, double *elbo, double *ll, double *lpj,
                   double *grad, double *f_out)
{
    orc_elbo_grad_ex(K, off, pos, inten, N, x, y, bg, pr, NULL, S, loc, raw, eps, elbo, ll, lpj, grad, f_out);
}

/*
 * Shared-shape estimator (Reading: one draw of the shape parameters per step
 * for all samples, each sample its own intensity): the noise of the shapes
 * j = 1..4 of every sample becomes sample 0's.  The estimator of the ELBO is
 * the plain one on this noise, so it stays unbiased; only its variance
 * changes.
 */
void orc_tie_shapes(int S, int K, double *eps)
{
    for (int s = 1; s < S; ++s)
        for (int k = 0; k < K; ++k)
            for (int j = 1; j < 5; ++j) eps[((size_t)s * K + k) * 5 + j] = eps[(size_t)k * 5 + j];
}

/* ------------------------------------------------------------------------ */
/* Optimiser (Reading: the paper names a gradient method; Adam is used)       */
/* ------------------------------------------------------------------------ */
/*
 * One Adam step (Kingma & Ba, 2015) minimising -ELBO: with gradient a = -grad,
 *   m <- b1 m + (1-b1) a;  v <- b2 v + (1-b2) a^2;
 *   p <- p - lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
 * params[K*10] = (loc[k][0..4], raw[k][0..4]) per phase.
 */
void orc_adam_step(int n, double *params, const double *grad, double *m, double *v, int t,
                   double lr, double b1, double b2, double eps)
{
    double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
    for (int i = 0; i < n; ++i) {
        double a = -grad[i];
        m[i] = b1 * m[i] + (1.0 - b1) * a;
        v[i] = b2 * v[i] + (1.0 - b2) * a * a;
        params[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}

/*
 * Stochastic variational inference: `iters` Adam steps on the ELBO, with the
 * noise of step t drawn by orc_normals(seed, 0, t0 + t, ...).  loc/raw ([K*5])
 * are updated in place; m, v ([K*10], layout as grad) carry the Adam moments;
 * t0 is the number of steps already taken.  trace[iters] receives the ELBO
 * estimate of each step (evaluated before that step's update).  orc_fit_ex
 * takes the variants as orc_elbo_grad_ex does (trace then holds that
 * objective; shared: the noise of orc_tie_shapes; bgfit: beta and its Adam
 * moments m_beta, v_beta are updated in place by the same step rule).
 */
void orc_fit_ex(int K, const int *off, const double *pos, const double *inten,
                int N, const double *x, const double *y, const double *bg,
                const orc_prior *pr, const orc_variant *var, int S, uint64_t seed, int t0, int iters,
                double lr, double b1, double b2, double adam_eps,
                double *loc, double *raw, double *m, double *v, double *trace)
{
    double *eps = (double *)malloc((size_t)S * K * 5 * sizeof(double));
    double *grad = (double *)malloc((size_t)K * 10 * sizeof(double));
    double *par = (double *)malloc((size_t)K * 10 * sizeof(double));
    double *gnoise = (double *)malloc((size_t)S * K * sizeof(double));
    double *ggate = (double *)malloc((size_t)K * sizeof(double));
    for (int t = 0; t < iters; ++t) {
        orc_normals(seed, 0u, (uint32_t)(t0 + t), S, K, eps);
        if (var && var->shared) orc_tie_shapes(S, K, eps);
        if (var && var->gates) orc_gate_noise(seed, 0u, (uint32_t)(t0 + t), S, K, gnoise);
        double elbo;
        double gb[3] = {0.0, 0.0, 0.0};
        orc_variant v2;
        if (var) { v2 = *var; v2.grad_beta = gb; v2.grad_gate = ggate; v2.gate_noise = gnoise; }
        orc_elbo_grad_ex(K, off, pos, inten, N, x, y, bg, pr, var ? &v2 : NULL, S, loc, raw, eps, &elbo, NULL, NULL,
                         grad, NULL);
        if (trace) trace[t] = elbo;
        if (var && var->bgfit)   /* the background coefficients take the same Adam step rule */
            orc_adam_step(3, var->beta, gb, var->m_beta, var->v_beta, t0 + t + 1, lr, b1, b2, adam_eps);
        if (var && var->gates)   /* and so do the gate logits */
            orc_adam_step(K, var->gate_a, ggate, var->m_gate, var->v_gate, t0 + t + 1, lr, b1, b2, adam_eps);
        for (int k = 0; k < K; ++k)
            for (int j = 0; j < 5; ++j) {
                par[k * 10 + j] = loc[k * 5 + j];
                par[k * 10 + 5 + j] = raw[k * 5 + j];
            }
        orc_adam_step(K * 10, par, grad, m, v, t0 + t + 1, lr, b1, b2, adam_eps);
        for (int k = 0; k < K; ++k)
            for (int j = 0; j < 5; ++j) {
                loc[k * 5 + j] = par[k * 10 + j];
                raw[k * 5 + j] = par[k * 10 + 5 + j];
            }
    }
    free(eps); free(grad); free(par); free(gnoise); free(ggate);
}

void orc_fit(int K, const int *off, const double *pos, const double *inten,
             int N, const double *x, const double *y, const double *bg,
             const orc_prior *pr, int S, uint64_t seed, int t0, int iters,
             double lr, double b1, double b2, double adam_eps,
             double *loc, double *raw, double *m, double *v, double *trace)
{
    orc_fit_ex(K, off, pos, inten, N, x, y, bg, pr, NULL, S, seed, t0, iters, lr, b1, b2, adam_eps,
               loc, raw, m, v, trace);
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
