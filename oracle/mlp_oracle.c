/*
 * mlp_oracle.c -- plain FP64 CPU reference of the learned star-pressure
 * guess: a 6 -> 64 -> 64 -> 1 perceptron with GELU activations that predicts
 * the star-region pressure p* of the exact Riemann solver (Sec. 2.1: Godunov
 * fluxes from the exact solution of the face Riemann problem) as the starting
 * point of its Newton iteration.
 *
 * TEST INFRASTRUCTURE ONLY, like fv_oracle.c: only the tests, the smoke check
 * and the CPU legs of the benchmark load it.  It shares no code with the CUDA
 * path.  The paper fixes none of this (it has no learned component); the
 * definitions below are the stated readings:
 *   features  the left and right states normalised by the pair's mean state:
 *             rbar, ubar, pbar the means of density, face-normal velocity and
 *             pressure, abar = sqrt(g pbar / rbar);
 *             x = ((rL-rbar)/rbar, (uL-ubar)/abar, (pL-pbar)/pbar,
 *                  (rR-rbar)/rbar, (uR-ubar)/abar, (pR-pbar)/pbar)
 *             (deviations, so that bfloat16 keeps 2^-9 of a small jump);
 *   targets   log(p* / pbar) (target 0), or log(p* / p_TR) / s(q) (target 1)
 *             with p_TR the two-rarefaction guess (Toro ch. 4), q = p_TR /
 *             min(pL, pR) - 1 its shock strength and s(q) = q^3 / (1 + q)^3
 *             for q > 0 (the guess is exact for two rarefactions, q <= 0,
 *             where the target is 0; its error is third order in a weak
 *             shock's strength and bounded for strong ones);
 *   GELU      tanh form, gelu(x) = x/2 (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3)));
 *   loss      mean over the samples of (y - t)^2;
 *   Adam      Kingma & Ba, bias-corrected moments.
 * Parameter layout (4673 values): W1[64][6], b1[64], W2[64][64], b2[64],
 * w3[64], b3 -- rows are output units.
 *
 * Pins (tests/test_oracle_mlp.py): gelu(x) - gelu(-x) = x; gelu'(0) = 1/2 and
 * the derivative against differences; a network built from mirrored unit
 * pairs computes a known affine map exactly; gradients against central
 * differences; the first two Adam steps against their closed forms;
 * features of mirrored states; the Sod star pressure of Toro's table; the
 * target of two rarefactions is 0 and the weak-shock scaling keeps the
 * target bounded as the shock vanishes.  tests/test_oracle_mutants.py plants
 * one plausible mistake at a time in a copy of this file and checks that
 * some pin fails.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define H 64
#define NIN 6
#define OFF_W1 0
#define OFF_B1 (OFF_W1 + H * NIN)
#define OFF_W2 (OFF_B1 + H)
#define OFF_B2 (OFF_W2 + H * H)
#define OFF_W3 (OFF_B2 + H)
#define OFF_B3 (OFF_W3 + H)
#define NPARAM (OFF_B3 + 1)

int orc_mlp_n_params(void) { return NPARAM; }

static const double K_GELU = 0.7978845608028654; /* sqrt(2/pi) */
static const double C_GELU = 0.044715;

double orc_gelu(double x) {
  double u = K_GELU * (x + C_GELU * x * x * x);
  return 0.5 * x * (1.0 + tanh(u));
}

/* d/dx of the tanh form: 1/2 (1 + tanh u) + x/2 (1 - tanh^2 u) du/dx */
double orc_gelu_grad(double x) {
  double u = K_GELU * (x + C_GELU * x * x * x);
  double th = tanh(u);
  double du = K_GELU * (1.0 + 3.0 * C_GELU * x * x);
  return 0.5 * (1.0 + th) + 0.5 * x * (1.0 - th * th) * du;
}

/* two-rarefaction guess of p* (Toro ch. 4), general gamma */
double orc_tr_guess(double gamma, double rL, double uL, double pL, double rR, double uR, double pR) {
  double z = (gamma - 1.0) / (2.0 * gamma);
  double aL = sqrt(gamma * pL / rL), aR = sqrt(gamma * pR / rR);
  double num = aL + aR - 0.5 * (gamma - 1.0) * (uR - uL);
  double den = aL / pow(pL, z) + aR / pow(pR, z);
  return pow(num / den, 1.0 / z);
}

/* pair = (rL, uL, pL, rR, uR, pR), face-normal velocities */
int orc_mlp_features(double gamma, const double *pair, double *x, double *pbar, double *ptr) {
  double rb = 0.5 * (pair[0] + pair[3]);
  double ub = 0.5 * (pair[1] + pair[4]);
  double pb = 0.5 * (pair[2] + pair[5]);
  double ab = sqrt(gamma * pb / rb);
  x[0] = (pair[0] - rb) / rb;
  x[1] = (pair[1] - ub) / ab;
  x[2] = (pair[2] - pb) / pb;
  x[3] = (pair[3] - rb) / rb;
  x[4] = (pair[4] - ub) / ab;
  x[5] = (pair[5] - pb) / pb;
  *pbar = pb;
  *ptr = orc_tr_guess(gamma, pair[0], pair[1], pair[2], pair[3], pair[4], pair[5]);
  return 0;
}

/* scale of the two-rarefaction guess's error: s(q) = (q / (1 + q))^3 for
 * q > 0, else 0 */
double orc_shock_scale(double q) {
  if (!(q > 0.0)) return 0.0;
  double r = q / (1.0 + q);
  return r * r * r;
}

/* training target of a pair with exact star pressure ps; *q_out the shock
 * strength of the two-rarefaction estimate */
double orc_mlp_target(double gamma, const double *pair, int target, double ps, double *q_out) {
  double x[NIN], pb, ptr;
  orc_mlp_features(gamma, pair, x, &pb, &ptr);
  double q = ptr / fmin(pair[2], pair[5]) - 1.0;
  if (q_out) *q_out = q;
  if (target == 0) return log(ps / pb);
  double sc = orc_shock_scale(q);
  return sc > 0.0 ? log(ps / ptr) / sc : 0.0;
}

/* one sample, FP64; keeps the pre-activations for the backward pass */
static double forward1(const double *th, const double *x, double *a1, double *h1, double *a2,
                       double *h2) {
  for (int o = 0; o < H; ++o) {
    double s = th[OFF_B1 + o];
    for (int i = 0; i < NIN; ++i) s += th[OFF_W1 + o * NIN + i] * x[i];
    a1[o] = s;
    h1[o] = orc_gelu(s);
  }
  for (int o = 0; o < H; ++o) {
    double s = th[OFF_B2 + o];
    for (int i = 0; i < H; ++i) s += th[OFF_W2 + o * H + i] * h1[i];
    a2[o] = s;
    h2[o] = orc_gelu(s);
  }
  double y = th[OFF_B3];
  for (int i = 0; i < H; ++i) y += th[OFF_W3 + i] * h2[i];
  return y;
}

int orc_mlp_forward(const double *theta, const double *x, int64_t n, double *y) {
  for (int64_t s = 0; s < n; ++s) {
    double a1[H], h1[H], a2[H], h2[H];
    y[s] = forward1(theta, x + NIN * s, a1, h1, a2, h2);
  }
  return 0;
}

/* round-to-nearest-even to bfloat16 (the upper 16 bits of a binary32),
 * from the definition: add half an ulp of the kept part (minus one when the
 * kept part is even, so ties go to even) and truncate.  Finite inputs. */
static float to_bf16(float v) {
  uint32_t u;
  memcpy(&u, &v, 4);
  u += 0x7fffu + ((u >> 16) & 1u);
  u &= 0xffff0000u;
  memcpy(&v, &u, 4);
  return v;
}

double orc_bf16_round(double v) { return (double)to_bf16((float)v); }

/* the quantised forward pass of the fused inference: inputs, W1, W2 and the
 * first hidden layer's activations rounded to bfloat16 (through binary32),
 * biases, the second hidden layer and the output layer kept in binary32
 * values; all sums and activations here in FP64 */
int orc_mlp_forward_bf16(const float *theta, const float *x, int64_t n, double *y) {
  for (int64_t s = 0; s < n; ++s) {
    double xq[NIN], h1[H];
    for (int i = 0; i < NIN; ++i) xq[i] = (double)to_bf16(x[NIN * s + i]);
    for (int o = 0; o < H; ++o) {
      double a = (double)theta[OFF_B1 + o];
      for (int i = 0; i < NIN; ++i) a += (double)to_bf16(theta[OFF_W1 + o * NIN + i]) * xq[i];
      h1[o] = (double)to_bf16((float)orc_gelu(a));
    }
    double out = (double)theta[OFF_B3];
    for (int o = 0; o < H; ++o) {
      double a = (double)theta[OFF_B2 + o];
      for (int i = 0; i < H; ++i) a += (double)to_bf16(theta[OFF_W2 + o * H + i]) * h1[i];
      out += (double)theta[OFF_W3 + o] * orc_gelu(a);
    }
    y[s] = out;
  }
  return 0;
}

/* loss = (1/n) sum_s (y_s - t_s)^2 and its gradient by the chain rule,
 * sample by sample in order */
int orc_mlp_loss_grad(const double *theta, const double *x, const double *t, int64_t n,
                      double *grad, double *loss) {
  if (n <= 0) return -1;
  memset(grad, 0, sizeof(double) * NPARAM);
  double L = 0.0;
  for (int64_t s = 0; s < n; ++s) {
    const double *xs = x + NIN * s;
    double a1[H], h1[H], a2[H], h2[H], d2[H], d1[H];
    double y = forward1(theta, xs, a1, h1, a2, h2);
    double e = y - t[s];
    L += e * e;
    double dy = 2.0 * e / (double)n;
    grad[OFF_B3] += dy;
    for (int i = 0; i < H; ++i) {
      grad[OFF_W3 + i] += dy * h2[i];
      d2[i] = dy * theta[OFF_W3 + i] * orc_gelu_grad(a2[i]);
    }
    for (int o = 0; o < H; ++o) {
      grad[OFF_B2 + o] += d2[o];
      for (int i = 0; i < H; ++i) grad[OFF_W2 + o * H + i] += d2[o] * h1[i];
    }
    for (int i = 0; i < H; ++i) {
      double s1 = 0.0;
      for (int o = 0; o < H; ++o) s1 += theta[OFF_W2 + o * H + i] * d2[o];
      d1[i] = s1 * orc_gelu_grad(a1[i]);
    }
    for (int o = 0; o < H; ++o) {
      grad[OFF_B1 + o] += d1[o];
      for (int i = 0; i < NIN; ++i) grad[OFF_W1 + o * NIN + i] += d1[o] * xs[i];
    }
  }
  *loss = L / (double)n;
  return 0;
}

/* one Adam step (step = 1, 2, ...):
 *   m <- b1 m + (1-b1) g,  v <- b2 v + (1-b2) g^2,
 *   theta <- theta - lr (m / (1-b1^step)) / (sqrt(v / (1-b2^step)) + eps) */
int orc_adam_step(double *theta, double *m, double *v, const double *grad, int64_t np, int step,
                  double lr, double b1, double b2, double eps) {
  if (step < 1) return -1;
  double c1 = 1.0 - pow(b1, step), c2 = 1.0 - pow(b2, step);
  for (int64_t k = 0; k < np; ++k) {
    m[k] = b1 * m[k] + (1.0 - b1) * grad[k];
    v[k] = b2 * v[k] + (1.0 - b2) * grad[k] * grad[k];
    theta[k] -= lr * (m[k] / c1) / (sqrt(v[k] / c2) + eps);
  }
  return 0;
}
