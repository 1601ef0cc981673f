// fv_riemann.cuh -- exact Godunov flux for the Euler equations on the GPU,
// templated on the arithmetic type (double: FP64 mode, float: FP32-flux
// mode).
//
// The paper (Sec. 2.1) computes face fluxes with Godunov's method, i.e. from
// the solution of the Riemann problem between the two face states.  The
// exact solver follows the published construction (Toro, "Riemann Solvers
// and Numerical Methods for Fluid Dynamics", ch. 4): pressure functions f_K
// (shock branch for p > p_K, rarefaction branch otherwise), Newton on
// f_L(p) + f_R(p) + (u_R - u_L) = 0 from the two-rarefaction guess (or a
// learned guess, see fv_mlp.cuh), the solution sampled on the face
// (x/t = 0).  Written from the equations.
#pragma once

#include <cuda_runtime.h>

namespace fvk {

template <typename T>
struct GasT {
  T g, gm1, gp1;
  T k_gm1_gp1;    // (g-1)/(g+1)
  T z;            // (g-1)/(2g)
  T inv_z;        // 2g/(g-1)
  T two_gm1;      // 2/(g-1)
  T shock_a;      // (g+1)/(2g)
  T shock_b;      // (g-1)/(2g)
  T inv_g;        // 1/g
  T tol;
  int maxit;
  __host__ __device__ static GasT make(double gamma, double tol, int maxit) {
    GasT G;
    G.g = (T)gamma;
    G.gm1 = (T)(gamma - 1.0);
    G.gp1 = (T)(gamma + 1.0);
    G.k_gm1_gp1 = (T)((gamma - 1.0) / (gamma + 1.0));
    G.z = (T)((gamma - 1.0) / (2.0 * gamma));
    G.inv_z = (T)(2.0 * gamma / (gamma - 1.0));
    G.two_gm1 = (T)(2.0 / (gamma - 1.0));
    G.shock_a = (T)((gamma + 1.0) / (2.0 * gamma));
    G.shock_b = (T)((gamma - 1.0) / (2.0 * gamma));
    G.inv_g = (T)(1.0 / gamma);
    G.tol = (T)tol;
    G.maxit = maxit;
    return G;
  }
};

__device__ __forceinline__ double fpow(double a, double b) { return pow(a, b); }
__device__ __forceinline__ float fpow(float a, float b) { return powf(a, b); }
__device__ __forceinline__ double fsqrt(double a) { return sqrt(a); }
// FP32: the square root as a product with the hardware reciprocal square
// root (about 2 ulps, two instructions instead of the correctly rounded
// sequence); every argument here is a positive finite sound speed or shock
// factor
__device__ __forceinline__ float fsqrt(float a) { return a * rsqrtf(a); }
// quotient inside the solver: exact in FP64; in FP32 the fast division
// intrinsic (a reciprocal and a product, about 2 ulps), well inside the
// FP32-flux mode's stated tolerance and its Newton stopping tests
__device__ __forceinline__ double qdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float qdiv(float a, float b) { return __fdividef(a, b); }

// pressure function of side K and its derivative (Toro Eqs. 4.6-4.7, 4.37)
template <typename T>
__device__ __forceinline__ void pressure_fn(const GasT<T> &G, T p, T rK, T pK, T aK, T &f, T &df) {
  if (p > pK) {
    T A = qdiv(T(2), G.gp1 * rK);
    T B = G.k_gm1_gp1 * pK;
    T q = fsqrt(qdiv(A, p + B));
    f = (p - pK) * q;
    df = q * (T(1) - qdiv(T(0.5) * (p - pK), B + p));
  } else {
    T pr = qdiv(p, pK);
    T pz = fpow(pr, G.z);
    f = (G.two_gm1 * aK) * (pz - T(1));
    // d/dp of the rarefaction branch: (p/pK)^(-(g+1)/(2g)) / (rK aK), and
    // -(g+1)/(2g) = z - 1
    df = qdiv(qdiv(pz, pr), rK * aK);
  }
}

// FP32 only: Newton has reached the precision floor when f = f_L + f_R + du
// is within a few ulps of its terms.  Near vacuum (p* much smaller than the
// flow's pressure scale) the terms cancel almost exactly and single-precision
// rounding of f alone moves the iterate by more than the relative-change
// tolerance, so that test could never pass.  FP64 keeps the plain
// relative-change test.
__device__ __forceinline__ bool at_rounding_floor(double, double, double, double) { return false; }
__device__ __forceinline__ bool at_rounding_floor(float f, float a, float b, float c) {
  return fabsf(f) <= 8.0f * 1.1920929e-7f * (fabsf(a) + fabsf(b) + fabsf(c));
}

// Star pressure/velocity.  Returns 0, or 1 (vacuum), 2 (no convergence).
// Newton starts from the two-rarefaction guess, or with GUESS from gabs when
// that is a positive finite pressure, else from the two-rarefaction guess
// times gmul (a learned correction factor, 1 when there is none).
template <typename T, bool GUESS = false>
__device__ __forceinline__ int riemann_star(const GasT<T> &G, T rL, T uL, T pL, T rR, T uR, T pR,
                                            T &ps, T &us, int &iters, T gabs = T(0),
                                            T gmul = T(1)) {
  T aL = fsqrt(qdiv(G.g * pL, rL)), aR = fsqrt(qdiv(G.g * pR, rR));
  T du = uR - uL;
  if (G.two_gm1 * (aL + aR) <= du) return 1;
  T p;
  if (GUESS && gabs > T(0) && isfinite(gabs)) {
    p = gabs;
  } else {
    T num = aL + aR - T(0.5) * G.gm1 * du;
    T den = qdiv(aL, fpow(pL, G.z)) + qdiv(aR, fpow(pR, G.z));
    p = fpow(qdiv(num, den), G.inv_z);
    if (GUESS) p *= gmul;
  }
  T pfloor = T(1e-6) * (pL < pR ? pL : pR);
  if (p < pfloor) p = pfloor;
  int it;
  bool conv = false;
  // as in riemann_star14: FP64 evaluates again at the final p, FP32 extends
  // the last values along their slopes
  T fL = T(0), fR = T(0), dfL = T(0), dfR = T(0), dp = T(0);
  for (it = 1; it <= G.maxit; ++it) {
    pressure_fn(G, p, rL, pL, aL, fL, dfL);
    pressure_fn(G, p, rR, pR, aR, fR, dfR);
    T fsum = fL + fR + du;
    if (at_rounding_floor(fsum, fL, fR, du)) {
      conv = true;
      dp = T(0);
      break;
    }
    T pn = p - qdiv(fsum, dfL + dfR);
    if (pn < pfloor) pn = pfloor;
    T change = qdiv(fabs(pn - p), T(0.5) * (pn + p));
    dp = pn - p;
    p = pn;
    if (change <= G.tol) {
      conv = true;
      break;
    }
  }
  iters = it;
  if (!conv || !(p > T(0)) || !isfinite(p)) return 2;
  if (sizeof(T) == 8) {
    pressure_fn(G, p, rL, pL, aL, fL, dfL);
    pressure_fn(G, p, rR, pR, aR, fR, dfR);
  } else {
    fL += dfL * dp;
    fR += dfR * dp;
  }
  ps = p;
  us = T(0.5) * (uL + uR) + T(0.5) * (fR - fL);
  return 0;
}

// the state on the face (x/t = 0) of the Riemann solution; side 0 = left of
// the contact (u* >= 0), 1 = right
template <typename T>
__device__ __forceinline__ void sample_face(const GasT<T> &G, T rL, T uL, T pL, T rR, T uR, T pR,
                                            T ps, T us, T &r, T &u, T &p, int &side) {
  if (T(0) <= us) {
    side = 0;
    T aL = fsqrt(qdiv(G.g * pL, rL));
    if (ps > pL) {
      T SL = uL - aL * fsqrt(G.shock_a * qdiv(ps, pL) + G.shock_b);
      if (T(0) <= SL) {
        r = rL; u = uL; p = pL;
      } else {
        T q = qdiv(ps, pL);
        r = rL * qdiv(q + G.k_gm1_gp1, G.k_gm1_gp1 * q + T(1));
        u = us; p = ps;
      }
    } else {
      T SHL = uL - aL;
      if (T(0) <= SHL) {
        r = rL; u = uL; p = pL;
      } else {
        T pr = qdiv(ps, pL);
        T STL = us - aL * fpow(pr, G.z);
        if (T(0) >= STL) {
          r = rL * fpow(pr, G.inv_g);
          u = us; p = ps;
        } else {
          T c = qdiv(T(2), G.gp1) + qdiv(G.gm1, G.gp1 * aL) * uL;
          r = rL * fpow(c, G.two_gm1);
          u = qdiv(T(2), G.gp1) * (aL + T(0.5) * G.gm1 * uL);
          p = pL * fpow(c, G.inv_z);
        }
      }
    }
  } else {
    side = 1;
    T aR = fsqrt(qdiv(G.g * pR, rR));
    if (ps > pR) {
      T SR = uR + aR * fsqrt(G.shock_a * qdiv(ps, pR) + G.shock_b);
      if (T(0) >= SR) {
        r = rR; u = uR; p = pR;
      } else {
        T q = qdiv(ps, pR);
        r = rR * qdiv(q + G.k_gm1_gp1, G.k_gm1_gp1 * q + T(1));
        u = us; p = ps;
      }
    } else {
      T SHR = uR + aR;
      if (T(0) >= SHR) {
        r = rR; u = uR; p = pR;
      } else {
        T pr = qdiv(ps, pR);
        T STR = us + aR * fpow(pr, G.z);
        if (T(0) <= STR) {
          r = rR * fpow(pr, G.inv_g);
          u = us; p = ps;
        } else {
          T c = qdiv(T(2), G.gp1) - qdiv(G.gm1, G.gp1 * aR) * uR;
          r = rR * fpow(c, G.two_gm1);
          u = qdiv(T(2), G.gp1) * (-aR + T(0.5) * G.gm1 * uR);
          p = pR * fpow(c, G.inv_z);
        }
      }
    }
  }
}

// ----------------------------------------------------------------------
// gamma = 1.4: every exponent of the exact solver is a multiple of 1/7
// (z = (g-1)/(2g) = 1/7, 2g/(g-1) = 7, 2/(g-1) = 5, 1/g = 5/7, and
// -(g+1)/(2g) = -6/7), so all powers reduce to integer powers of the inverse
// seventh root r = x^(-1/7).  r comes from a single-precision seed refined by
// Newton's method on r^-7 = x, r <- r (8 - x r^7) / 7 (quadratic
// convergence: two steps take a ~1e-7 seed to double-precision rounding).
// Per Riemann problem: one root per side, one per Newton iterate (shared by
// both sides), one at the converged star pressure.

__device__ __forceinline__ double rroot7(double x) {
  double r = (double)exp2f(-0.14285714285714285f * __log2f((float)x));
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    double r2 = r * r, r4 = r2 * r2;
    double r7 = r4 * r2 * r;
    r = r * (8.0 - x * r7) * (1.0 / 7.0);
  }
  return r;
}
__device__ __forceinline__ float rroot7(float x) {
  float r = exp2f(-0.14285714285714285f * __log2f(x));
  float r2 = r * r, r4 = r2 * r2;
  return r * (8.0f - x * (r4 * r2 * r)) * (1.0f / 7.0f);
}
// FP32: the inverse seventh roots of two values at once, the Newton step
// with paired instructions (the seed's logarithm and power stay per value)
__device__ __forceinline__ float2 rroot7_pair(float2 x) {
  const float2 lg = __fmul2_rn(make_float2(__log2f(x.x), __log2f(x.y)),
                               make_float2(-0.14285714285714285f, -0.14285714285714285f));
  const float2 r = make_float2(exp2f(lg.x), exp2f(lg.y));
  const float2 r2 = __fmul2_rn(r, r), r4 = __fmul2_rn(r2, r2);
  const float2 r7 = __fmul2_rn(__fmul2_rn(r4, r2), r);
  const float2 t = __ffma2_rn(make_float2(-x.x, -x.y), r7, make_float2(8.0f, 8.0f));
  return __fmul2_rn(__fmul2_rn(r, t), make_float2(1.0f / 7.0f, 1.0f / 7.0f));
}

template <typename T>
__device__ __forceinline__ T ipow5(T c) {
  T c2 = c * c;
  return c2 * c2 * c;
}
template <typename T>
__device__ __forceinline__ T ipow7(T c) {
  T c2 = c * c, c4 = c2 * c2;
  return c4 * c2 * c;
}

// per-side constants: iq = pK^(-1/7); cK = pK iq / (rK aK) (rarefaction slope
// factor); eK = 2 aK / (g-1) = 5 aK
template <typename T>
struct Side14 {
  T r, p, a, iq, c, e, A, B;
};

template <typename T>
__device__ __forceinline__ Side14<T> make_side14(const GasT<T> &G, T rK, T pK) {
  Side14<T> s;
  s.r = rK;
  s.p = pK;
  s.a = fsqrt(qdiv(G.g * pK, rK));
  s.iq = rroot7(pK);
  s.c = qdiv(pK * s.iq, rK * s.a);
  s.e = T(5) * s.a;
  s.A = qdiv(T(2), G.gp1 * rK);
  s.B = G.k_gm1_gp1 * pK;
  return s;
}

// FP32: both sides' constants at once with paired instructions (the
// reciprocals, square roots and the seventh roots' seeds stay per side):
// a = sqrt(g p / r), iq = p^(-1/7), c = p iq / (r a), e = 5 a,
// A = 2 / ((g+1) r), B = (g-1)/(g+1) p
__device__ __forceinline__ void make_sides14_pair(const GasT<float> &G, float rL, float pL, float rR, float pR,
                                                  Side14<float> &L, Side14<float> &R) {
  const float2 p = make_float2(pL, pR), r = make_float2(rL, rR);
  const float2 ir = make_float2(qdiv(1.0f, rL), qdiv(1.0f, rR));
  const float2 q = __fmul2_rn(__fmul2_rn(make_float2(G.g, G.g), p), ir);
  const float2 a = __fmul2_rn(q, make_float2(rsqrtf(q.x), rsqrtf(q.y)));
  const float2 iq = rroot7_pair(p);
  const float2 ra = __fmul2_rn(r, a);
  const float2 c = __fmul2_rn(__fmul2_rn(p, iq), make_float2(qdiv(1.0f, ra.x), qdiv(1.0f, ra.y)));
  const float2 e = __fmul2_rn(make_float2(5.0f, 5.0f), a);
  const float two_gp1 = (float)(2.0 / (1.4 + 1.0));  // the gamma = 1.4 path only
  const float2 A = __fmul2_rn(make_float2(two_gp1, two_gp1), ir);
  const float2 B = __fmul2_rn(make_float2(G.k_gm1_gp1, G.k_gm1_gp1), p);
  L.r = rL;
  L.p = pL;
  L.a = a.x;
  L.iq = iq.x;
  L.c = c.x;
  L.e = e.x;
  L.A = A.x;
  L.B = B.x;
  R.r = rR;
  R.p = pR;
  R.a = a.y;
  R.iq = iq.y;
  R.c = c.y;
  R.e = e.y;
  R.A = A.y;
  R.B = B.y;
}

// f_K(p) and f_K'(p), one branch each: shock14 for p > pK, rare14 otherwise
// (Toro Eqs. 4.6-4.7, 4.37).  The rarefaction branch in FP64 comes from
// p17 = p^(1/7) and rp6 = p^(-6/7), shared by both sides; in FP32 from the
// root of p/pK itself, with (p/pK)^(1/7) taken as the reciprocal of the
// inverse root (about one ulp), which keeps f_K smooth enough for Newton's
// stopping test; forming it as a product with the sixth power of the root
// would multiply the single-precision error by six.
__device__ __forceinline__ void shock14(const Side14<double> &K, double p, double &f, double &df) {
  double q = sqrt(K.A / (p + K.B));
  f = (p - K.p) * q;
  df = q * (1.0 - 0.5 * (p - K.p) / (K.B + p));
}
__device__ __forceinline__ void shock14(const Side14<float> &K, float p, float &f, float &df) {
  float q = fsqrt(qdiv(K.A, p + K.B));
  f = (p - K.p) * q;
  df = q * (1.0f - qdiv(0.5f * (p - K.p), K.B + p));
}
__device__ __forceinline__ void rare14(const Side14<double> &K, double, double p17, double rp6,
                                       double &f, double &df) {
  f = K.e * (p17 * K.iq - 1.0);
  df = K.c * rp6;
}
__device__ __forceinline__ void rare14(const Side14<float> &K, float p, float, float, float &f,
                                       float &df) {
  float pr = qdiv(p, K.p);
  float ir = rroot7(pr);             // pr^(-1/7), about one ulp
  float ir2 = ir * ir;
  float ir6 = ir2 * ir2 * ir2;       // pr^(-6/7), only the slope uses it
  f = K.e * (qdiv(1.0f, ir) - 1.0f);  // pr^(1/7) - 1 from the reciprocal
  df = qdiv(ir6, K.r * K.a);
}

// f_L, f_L', f_R, f_R' at p, the branches sorted across the two sides: a
// lane runs the shock formula once per side on its shock branch and the
// rarefaction formula once per side on its rarefaction branch, on that
// side's constants taken by selection.  A warp whose lanes differ in which
// side is on which branch (the usual case: the star pressure lies between
// pL and pR, and a face's orientation decides which side is the higher)
// runs each formula once instead of each formula once per side.  Every
// value is the one the branch computes for that side alone.
template <typename T>
__device__ __forceinline__ void pressure_fns14(const Side14<T> &L, const Side14<T> &R, T p, T p17,
                                               T rp6, T &fL, T &dfL, T &fR, T &dfR) {
  const bool sL = p > L.p, sR = p > R.p;
  T f, df;
  if (sL || sR) {
    const Side14<T> K = sL ? L : R;
    shock14(K, p, f, df);
    if (sL) {
      fL = f;
      dfL = df;
    } else {
      fR = f;
      dfR = df;
    }
  }
  if (sL && sR) shock14(R, p, fR, dfR);
  if (!(sL && sR)) {
    const Side14<T> K = sL ? R : L;
    rare14(K, p, p17, rp6, f, df);
    if (sL) {
      fR = f;
      dfR = df;
    } else {
      fL = f;
      dfL = df;
    }
  }
  if (!(sL || sR)) rare14(R, p, p17, rp6, fR, dfR);
}

// (ps/pK)^(1/7) for the sampling step, on the rarefaction branch of side K.
// FP64: p17 (K.iq = pK^(-1/7)).  FP32: from the side's pressure function at
// ps, fK = eK ((ps/pK)^(1/7) - 1), which Newton has already formed, instead
// of another seventh root: 1 + fK/eK carries fK's few-ulp error only in
// the difference from 1, so it is at least as close as a root taken anew
// (the one-step extension of fK to ps neglects ~1e-12 relative).
__device__ __forceinline__ double ratio17(const Side14<double> &K, double p17, double) {
  return p17 * K.iq;
}
__device__ __forceinline__ float ratio17(const Side14<float> &K, float, float fK) {
  return 1.0f + qdiv(fK, K.e);
}

template <typename T>
__device__ __forceinline__ void roots_of(T p, T &p17, T &rp6) {
  T rp = rroot7(p);
  T rp2 = rp * rp;
  rp6 = rp2 * rp2 * rp2;
  p17 = p * rp6;
}

template <typename T, bool GUESS = false>
__device__ __forceinline__ int riemann_star14(const GasT<T> &G, const Side14<T> &L, T uL,
                                              const Side14<T> &R, T uR, T &ps, T &us, T &ps17,
                                              T &fLs, T &fRs, int &iters, T gabs = T(0),
                                              T gmul = T(1)) {
  T du = uR - uL;
  if (G.two_gm1 * (L.a + R.a) <= du) return 1;
  T p;
  if (GUESS && gabs > T(0) && isfinite(gabs)) {
    p = gabs;
  } else {
    T num = L.a + R.a - T(0.5) * G.gm1 * du;
    p = ipow7(qdiv(num, L.a * L.iq + R.a * R.iq));
    if (GUESS) p *= gmul;
  }
  T pfloor = T(1e-6) * (L.p < R.p ? L.p : R.p);
  if (p < pfloor) p = pfloor;
  int it;
  bool conv = false;
  // fL, fR and their slopes at the last evaluated iterate, and the step from
  // it to the final p (0 on the rounding-floor exit).  FP64 evaluates both
  // pressure functions again at the final p, as the oracle does.  FP32
  // extends the last values to it along their slopes: the FP32 tolerance
  // (2e-6) bounds the step, so the neglected second-order term is ~1e-12
  // relative, far below single-precision rounding, and the two evaluations
  // are saved.
  T fL = T(0), fR = T(0), dfL = T(0), dfR = T(0), dp = T(0);
  for (it = 1; it <= G.maxit; ++it) {
    T p17 = T(0), rp6 = T(0);
    if (sizeof(T) == 8 && (p <= L.p || p <= R.p)) roots_of(p, p17, rp6);
    pressure_fns14(L, R, p, p17, rp6, fL, dfL, fR, dfR);
    T fsum = fL + fR + du;
    if (at_rounding_floor(fsum, fL, fR, du)) {
      conv = true;
      dp = T(0);
      break;
    }
    T pn = p - qdiv(fsum, dfL + dfR);
    if (pn < pfloor) pn = pfloor;
    T change = qdiv(fabs(pn - p), T(0.5) * (pn + p));
    dp = pn - p;
    p = pn;
    if (change <= G.tol) {
      conv = true;
      break;
    }
  }
  iters = it;
  if (!conv || !(p > T(0)) || !isfinite(p)) return 2;
  T p17 = T(0), rp6 = T(0);
  if (sizeof(T) == 8) {
    roots_of(p, p17, rp6);
    pressure_fns14(L, R, p, p17, rp6, fL, dfL, fR, dfR);
  } else {
    fL += dfL * dp;
    fR += dfR * dp;
  }
  ps = p;
  ps17 = p17;
  fLs = fL;
  fRs = fR;
  us = T(0.5) * (uL + uR) + T(0.5) * (fR - fL);
  return 0;
}

// the state on the face (x/t = 0); p17 = ps^(1/7), fL and fR the pressure
// functions at ps.  One code path for both
// sides: the sampled side K (left when u* >= 0) is taken by selection, and
// on the right every velocity is mirrored (negated), which turns the right
// side's wave tests and fan formulas into the left side's; the face
// velocity is mirrored back at the end.  Negation is exact and rounding is
// symmetric in sign, so each value is the one the right side's own formulas
// give, while a warp whose faces sample both sides runs the formulas once.
template <typename T>
__device__ __forceinline__ void sample_face14(const GasT<T> &G, const Side14<T> &L, T uL,
                                              const Side14<T> &R, T uR, T ps, T us, T p17, T fL,
                                              T fR, T &r, T &u, T &p, int &side) {
  const bool left = T(0) <= us;
  side = left ? 0 : 1;
  const Side14<T> K = left ? L : R;
  const T fK = left ? fL : fR;
  const T uK = left ? uL : -uR;  // the side's velocity, mirrored on the right
  const T uS = left ? us : -us;  // u*, likewise
  T um;                          // the face velocity, mirrored on the right
  if (ps > K.p) {
    T SK = uK - K.a * fsqrt(G.shock_a * qdiv(ps, K.p) + G.shock_b);
    if (T(0) <= SK) {
      r = K.r; um = uK; p = K.p;
    } else {
      T q = qdiv(ps, K.p);
      r = K.r * qdiv(q + G.k_gm1_gp1, G.k_gm1_gp1 * q + T(1));
      um = uS; p = ps;
    }
  } else {
    T SHK = uK - K.a;
    if (T(0) <= SHK) {
      r = K.r; um = uK; p = K.p;
    } else {
      T pr17 = ratio17(K, p17, fK);  // (ps/pK)^(1/7)
      T STK = uS - K.a * pr17;
      if (T(0) >= STK) {
        r = K.r * ipow5(pr17);
        um = uS; p = ps;
      } else {
        T c = qdiv(T(2), G.gp1) + qdiv(G.gm1, G.gp1 * K.a) * uK;
        r = K.r * ipow5(c);
        um = qdiv(T(2), G.gp1) * (K.a + T(0.5) * G.gm1 * uK);
        p = K.p * ipow7(c);
      }
    }
  }
  u = left ? um : -um;
}

// the flux of a face whose Riemann problem failed (vacuum, or Newton did not
// converge): NaN, so that the failure reaches the state it would corrupt and
// the state check reports it, the same way whatever the registers held
template <typename T>
__device__ __forceinline__ void failed_flux(T F[5]) {
#pragma unroll
  for (int c = 0; c < 5; ++c) F[c] = (T)__int_as_float(0x7fc00000);
}

// Godunov flux per unit area through an interior face with unit normal n;
// the tangential velocity comes from the upwind side of the contact.
// Returns 0 or the riemann_star error.
template <typename T, bool G14, bool GUESS = false>
__device__ __forceinline__ int godunov_flux(const GasT<T> &G, const T WL[5], const T WR[5],
                                            const T n[3], T F[5], int &iters, T gabs = T(0),
                                            T gmul = T(1)) {
  T unL = (WL[1] * n[0] + WL[2] * n[1]) + WL[3] * n[2];
  T unR = (WR[1] * n[0] + WR[2] * n[1]) + WR[3] * n[2];
  T ps, us;
  T r0, un0, p0;
  int side;
  if (G14) {
    Side14<T> L, R;
    if constexpr (sizeof(T) == 4) {
      make_sides14_pair(G, WL[0], WL[4], WR[0], WR[4], L, R);
    } else {
      L = make_side14(G, WL[0], WL[4]);
      R = make_side14(G, WR[0], WR[4]);
    }
    T p17, fLs, fRs;
    int rc = riemann_star14<T, GUESS>(G, L, unL, R, unR, ps, us, p17, fLs, fRs, iters, gabs, gmul);
    if (rc) {
      failed_flux(F);
      return rc;
    }
    sample_face14(G, L, unL, R, unR, ps, us, p17, fLs, fRs, r0, un0, p0, side);
  } else {
    int rc = riemann_star<T, GUESS>(G, WL[0], unL, WL[4], WR[0], unR, WR[4], ps, us, iters, gabs,
                                    gmul);
    if (rc) {
      failed_flux(F);
      return rc;
    }
    sample_face(G, WL[0], unL, WL[4], WR[0], unR, WR[4], ps, us, r0, un0, p0, side);
  }
  const bool left = side == 0;
  T uns = left ? unL : unR;
  T V0[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) V0[d] = un0 * n[d] + ((left ? WL[1 + d] : WR[1 + d]) - uns * n[d]);
  T mass = r0 * un0;
  T E0 = qdiv(p0, G.gm1) + T(0.5) * r0 * ((V0[0] * V0[0] + V0[1] * V0[1]) + V0[2] * V0[2]);
  F[0] = mass;
#pragma unroll
  for (int d = 0; d < 3; ++d) F[1 + d] = mass * V0[d] + p0 * n[d];
  F[4] = un0 * (E0 + p0);
  return 0;
}

// Boundary fluxes: a slip wall solves (rho, u_n, p | rho, -u_n, p), whose
// contact speed is exactly 0, so only the star pressure crosses it; a
// transmissive face has identical states on both sides, whose Godunov flux
// is the physical flux.
template <typename T, bool G14>
__device__ __forceinline__ int boundary_flux(const GasT<T> &G, int bc, const T WL[5], const T n[3],
                                             T F[5], int &iters) {
  T un = (WL[1] * n[0] + WL[2] * n[1]) + WL[3] * n[2];
  if (bc == 1) {
    T ps, us;
    int rc;
    if (G14) {
      Side14<T> S = make_side14(G, WL[0], WL[4]);
      T p17, fLs, fRs;
      rc = riemann_star14(G, S, un, S, -un, ps, us, p17, fLs, fRs, iters);
    } else {
      rc = riemann_star(G, WL[0], un, WL[4], WL[0], -un, WL[4], ps, us, iters);
    }
    if (rc) {
      failed_flux(F);
      return rc;
    }
    F[0] = T(0);
    F[1] = ps * n[0];
    F[2] = ps * n[1];
    F[3] = ps * n[2];
    F[4] = T(0);
    return 0;
  }
  iters = 0;
  T r = WL[0], p = WL[4];
  T E = qdiv(p, G.gm1) + T(0.5) * r * ((WL[1] * WL[1] + WL[2] * WL[2]) + WL[3] * WL[3]);
  T mass = r * un;
  F[0] = mass;
#pragma unroll
  for (int d = 0; d < 3; ++d) F[1 + d] = mass * WL[1 + d] + p * n[d];
  F[4] = un * (E + p);
  return 0;
}

}  // namespace fvk
