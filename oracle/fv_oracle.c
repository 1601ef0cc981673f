/*
 * fv_oracle.c -- plain, slow FP64 CPU oracle of the temporally adaptive
 * explicit finite-volume solver (Couteyen Carpaye, Roman, Brenner 2017).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA path: it has its own face extraction, geometry, gradient,
 * limiter, Riemann solver and time-level schedule, written from the maths.
 *
 * What it computes (paper Sec. 2.2, Eq. 1 and Algorithm 2):
 *   - Eq. 1 with S = 0 and inviscid Euler fluxes (gamma from the config):
 *       d/dt (V_i U_i) = - sum_f sigma_f F_f A_f
 *   - Alg. 2, time steps: a local explicit time step per cell; Delta t = min.
 *   - Alg. 2, levels: level k_i with dt_k = 2^k Delta t, neighbours within 1.
 *   - Alg. 2, subiterations: 2^theta subiterations; level k begins every 2^k.
 *   - Predictor / corrector ("extensive prediction / correction"): one Heun
 *     (SSP-RK2) step per level step, fluxes in flux form; neighbours of other
 *     levels taken at the right time by linear interpolation in time
 *     ("repositioning / interpolation"); a coarse cell takes the time
 *     integral of the fine-side fluxes across a level interface.
 *   - Two orders of the level steps within a cycle: order 0 ends each level's
 *     step when its time is reached, finest first, the coarse cell taking the
 *     fine-side integrals across an interface at once; order 1 is the order
 *     of Alg. 2's loops (every level that begins at subiteration s is
 *     predicted and corrected in it, coarsest first, and its interface
 *     integrals are corrected when its next step begins -- Alg. 2's
 *     intensive correction; Alg. 3's extra subiteration applies the last).
 * Scheme choices the paper leaves open (the same on the CUDA path):
 *   least-squares gradients of primitives, MUSCL reconstruction with the
 *   minmod limiter, the exact Godunov Riemann solver (Toro, "Riemann Solvers
 *   and Numerical Methods for Fluid Dynamics", ch. 4: pressure functions,
 *   Newton iteration on p*, sampling at x/t = 0).
 *
 * Loops are in natural order; OpenMP is used only over independent items
 * (each iteration writes its own slot), so results do not depend on the
 * thread count.  Build with -ffp-contract=off.
 *
 * Pins (tests/test_oracle_pins.py; no function is unpinned):
 *   riemann_star, riemann_sample  Toro's Table 4.3 (p*, u* and the star
 *       densities of five tests); exact guess and one Newton iteration on
 *       two rarefactions; mirror symmetry of the sampled solution and its
 *       continuity at fan edges; Sod's self-similar profile; for several
 *       gamma the jump conditions of every wave (Rankine-Hugoniot across
 *       shocks, isentropic fans with their characteristic structure);
 *   godunov_flux, boundary_flux, ghost_state  identical states give the
 *       physical flux; supersonic flow is upwind; F(WL,WR,n) = -F(WR,WL,-n);
 *       a wall passes only the star pressure, equal to the Godunov flux
 *       against the reflected state; the ghost is a reflection (wall) or a
 *       copy (transmissive);
 *   muscl_pair, minmod  textbook 1D MUSCL-minmod on a uniform chain;
 *   gradient_cell and the weights  exact on linear fields;
 *   orc_create geometry  closed cells, total volume and surface, face
 *       count, centroid offsets and mirrored ghost centroids;
 *   local_dt, orc_assign_levels  numpy and a graph distance transform;
 *   phase_at, phase_at_paper  the tau(s) example of Sec. 2.2 and Alg. 2's
 *       loops; per-cycle update counts = C(tau) and the paper's Tables 1-3;
 *   the phases  free stream kept; conservation ledger to round-off (walls
 *       with a net impulse, open ends with through-flow; both orders); one
 *       level = global Heun stepping bitwise; Sod converges to the exact
 *       solution; better than first-order time consistency across levels;
 *       the two orders agree to O(dt^2); a begin phase's predictor equals
 *       the level residual at its time (first and later subiterations).
 * tests/test_oracle_mutants.py plants one plausible mistake at a time in a
 * copy of this file and checks that some pin fails.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXL 8

enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_EMESH = -2, ORC_ENONPHYS = -4, ORC_ERIEMANN = -5 };

static char g_msg[512];
static void set_msg(const char *s) {
  strncpy(g_msg, s, sizeof g_msg - 1);
  g_msg[sizeof g_msg - 1] = 0;
}
const char *orc_error(void) { return g_msg; }

/* ------------------------------------------------------------------ gas --- */
typedef struct {
  double g, gm1, gp1;
  double tol;
  int maxit;
} gas_t;

/* ------------------------------------------------------------- solver --- */
typedef struct orc {
  gas_t gas;
  double cfl;
  int L;     /* number of levels (max_levels) */
  int theta; /* L - 1 */
  int64_t nc, nf;
  /* cells (original tet order) */
  double *vol;     /* nc */
  double *xc;      /* 3 nc */
  int64_t *cface;  /* 4 nc: face id of local face j (face opposite node j) */
  int8_t *csgn;    /* 4 nc: +1 if the cell owns the face, -1 otherwise */
  double *lsw;     /* 12 nc: least-squares weights, 3 per local face */
  /* faces */
  int64_t *fown, *fnb; /* fnb = -1 on the boundary */
  int8_t *fbc;         /* 0 interior, 1 slip wall, 2 transmissive */
  double *farea, *fnrm, *fr; /* area; unit normal owner->outside; x_R - x_L */
  /* state */
  double *U, *Us;   /* 5 nc each: U^n and the predicted U* */
  double *W;        /* 5 nc primitives at the phase time */
  double *G;        /* 15 nc gradients, G[15 i + 3 c + d] */
  double *F1A;      /* 5 nf: F A at the step start, later Phi^step */
  double *ACC;      /* 5 nf: fine-side flux time integral on level interfaces */
  double *BND;      /* 5 nf: running boundary flux integral per face */
  double *dt;       /* nc */
  int8_t *lev, *flev;
  unsigned char *mark;
  double t, dtmin;
  int have_levels; /* 1 inside a cycle (levels assigned) */
  int order;       /* 0: corrector of the finest level first, at the end of its
                     step; 1: the paper's order (see phase_at_paper) */
  int next_phase;  /* index of the next phase inside the cycle */
  int64_t tn[ORC_MAXL]; /* step start of each level, in Delta t units */
  int pred[ORC_MAXL];   /* 1 while U* of that level is valid */
  /* statistics */
  int64_t n_updates[ORC_MAXL], n_faceevals[ORC_MAXL];
  int64_t newton_iters, riemann_calls;
} orc;

/* ============================================================ Riemann === */
/* Toro ch. 4, Eqs. (4.6)-(4.7) and their derivatives: the pressure
 * function of one side K and its slope.  p > pK: shock branch; otherwise
 * rarefaction branch. */
static void pressure_fn(const gas_t *G, double p, double rK, double pK, double aK, double *f,
                        double *df) {
  if (p > pK) {
    double A = 2.0 / (G->gp1 * rK);
    double B = (G->gm1 / G->gp1) * pK;
    double q = sqrt(A / (p + B));
    *f = (p - pK) * q;
    *df = q * (1.0 - 0.5 * (p - pK) / (B + p));
  } else {
    double pr = p / pK;
    double z = G->gm1 / (2.0 * G->g);
    *f = (2.0 * aK / G->gm1) * (pow(pr, z) - 1.0);
    *df = (1.0 / (rK * aK)) * pow(pr, -G->gp1 / (2.0 * G->g));
  }
}

/* Star pressure and velocity of the 1D Riemann problem (rL,uL,pL | rR,uR,pR).
 * Initial guess: two-rarefaction approximation (Toro Eq. 4.46).  Newton
 * iteration stops when the relative change |p_new - p| / (0.5 (p_new + p))
 * is <= tol; iterates are floored at 1e-6 min(pL, pR).  Returns
 * ORC_ERIEMANN on vacuum generation or non-convergence. */
static int riemann_star(const gas_t *G, double rL, double uL, double pL, double rR, double uR,
                        double pR, double *ps, double *us, int *iters) {
  double aL = sqrt(G->g * pL / rL), aR = sqrt(G->g * pR / rR);
  double du = uR - uL;
  if ((2.0 / G->gm1) * (aL + aR) <= du) return ORC_ERIEMANN; /* vacuum */
  double z = G->gm1 / (2.0 * G->g);
  double num = aL + aR - 0.5 * G->gm1 * du;
  double den = aL / pow(pL, z) + aR / pow(pR, z);
  double p = pow(num / den, 1.0 / z);
  double pfloor = 1e-6 * (pL < pR ? pL : pR);
  if (p < pfloor) p = pfloor;
  int it, conv = 0;
  for (it = 1; it <= G->maxit; ++it) {
    double fL, dfL, fR, dfR;
    pressure_fn(G, p, rL, pL, aL, &fL, &dfL);
    pressure_fn(G, p, rR, pR, aR, &fR, &dfR);
    double pn = p - (fL + fR + du) / (dfL + dfR);
    if (pn < pfloor) pn = pfloor;
    double change = fabs(pn - p) / (0.5 * (pn + p));
    p = pn;
    if (change <= G->tol) {
      conv = 1;
      break;
    }
  }
  if (!conv || !(p > 0.0) || !isfinite(p)) return ORC_ERIEMANN;
  double fL, dfL, fR, dfR;
  pressure_fn(G, p, rL, pL, aL, &fL, &dfL);
  pressure_fn(G, p, rR, pR, aR, &fR, &dfR);
  *ps = p;
  *us = 0.5 * (uL + uR) + 0.5 * (fR - fL);
  *iters = it;
  return ORC_OK;
}

/* Toro Sec. 4.5: the self-similar solution at speed xi = x/t.  *side is 0
 * when the sample lies left of the contact (xi <= u*), 1 otherwise. */
static void riemann_sample(const gas_t *G, double rL, double uL, double pL, double rR, double uR,
                           double pR, double ps, double us, double xi, double *r, double *u,
                           double *p, int *side) {
  double g = G->g, gm1 = G->gm1, gp1 = G->gp1;
  double aL = sqrt(g * pL / rL), aR = sqrt(g * pR / rR);
  if (xi <= us) {
    *side = 0;
    if (ps > pL) { /* left shock */
      double SL = uL - aL * sqrt((gp1 / (2.0 * g)) * (ps / pL) + gm1 / (2.0 * g));
      if (xi <= SL) {
        *r = rL; *u = uL; *p = pL;
      } else {
        double q = ps / pL, k = gm1 / gp1;
        *r = rL * ((q + k) / (k * q + 1.0));
        *u = us; *p = ps;
      }
    } else { /* left rarefaction */
      double SHL = uL - aL;
      if (xi <= SHL) {
        *r = rL; *u = uL; *p = pL;
      } else {
        double asL = aL * pow(ps / pL, gm1 / (2.0 * g));
        double STL = us - asL;
        if (xi >= STL) {
          *r = rL * pow(ps / pL, 1.0 / g);
          *u = us; *p = ps;
        } else { /* inside the fan */
          double c = 2.0 / gp1 + (gm1 / (gp1 * aL)) * (uL - xi);
          *r = rL * pow(c, 2.0 / gm1);
          *u = (2.0 / gp1) * (aL + 0.5 * gm1 * uL + xi);
          *p = pL * pow(c, 2.0 * g / gm1);
        }
      }
    }
  } else {
    *side = 1;
    if (ps > pR) { /* right shock */
      double SR = uR + aR * sqrt((gp1 / (2.0 * g)) * (ps / pR) + gm1 / (2.0 * g));
      if (xi >= SR) {
        *r = rR; *u = uR; *p = pR;
      } else {
        double q = ps / pR, k = gm1 / gp1;
        *r = rR * ((q + k) / (k * q + 1.0));
        *u = us; *p = ps;
      }
    } else { /* right rarefaction */
      double SHR = uR + aR;
      if (xi >= SHR) {
        *r = rR; *u = uR; *p = pR;
      } else {
        double asR = aR * pow(ps / pR, gm1 / (2.0 * g));
        double STR = us + asR;
        if (xi <= STR) {
          *r = rR * pow(ps / pR, 1.0 / g);
          *u = us; *p = ps;
        } else {
          double c = 2.0 / gp1 - (gm1 / (gp1 * aR)) * (uR - xi);
          *r = rR * pow(c, 2.0 / gm1);
          *u = (2.0 / gp1) * (-aR + 0.5 * gm1 * uR + xi);
          *p = pR * pow(c, 2.0 * g / gm1);
        }
      }
    }
  }
}

/* Godunov flux through a face with unit normal n, per unit area, in the
 * global frame: the 1D problem is solved along n; the tangential velocity is
 * carried from the upwind side of the contact (paper Sec. 2.1: "Godunov's
 * method for solving the Riemann problem"). */
static int godunov_flux(const gas_t *G, const double *WL, const double *WR, const double *n,
                        double *F, int *iters) {
  double unL = (WL[1] * n[0] + WL[2] * n[1]) + WL[3] * n[2];
  double unR = (WR[1] * n[0] + WR[2] * n[1]) + WR[3] * n[2];
  double ps, us;
  int rc = riemann_star(G, WL[0], unL, WL[4], WR[0], unR, WR[4], &ps, &us, iters);
  if (rc) return rc;
  double r0, un0, p0;
  int side;
  riemann_sample(G, WL[0], unL, WL[4], WR[0], unR, WR[4], ps, us, 0.0, &r0, &un0, &p0, &side);
  const double *Ws = side == 0 ? WL : WR;
  double uns = side == 0 ? unL : unR;
  double V0[3];
  for (int d = 0; d < 3; ++d) V0[d] = un0 * n[d] + (Ws[1 + d] - uns * n[d]);
  double mass = r0 * un0;
  double E0 = p0 / G->gm1 + 0.5 * r0 * ((V0[0] * V0[0] + V0[1] * V0[1]) + V0[2] * V0[2]);
  F[0] = mass;
  for (int d = 0; d < 3; ++d) F[1 + d] = mass * V0[d] + p0 * n[d];
  F[4] = un0 * (E0 + p0);
  return ORC_OK;
}

/* ========================================================= primitives === */
static void cons_to_prim(const gas_t *G, const double *U, double *W) {
  double r = U[0];
  double u = U[1] / r, v = U[2] / r, w = U[3] / r;
  double ke = 0.5 * r * ((u * u + v * v) + w * w);
  W[0] = r; W[1] = u; W[2] = v; W[3] = w;
  W[4] = G->gm1 * (U[4] - ke);
}

static void prim_to_cons(const gas_t *G, const double *W, double *U) {
  double r = W[0];
  U[0] = r;
  U[1] = r * W[1]; U[2] = r * W[2]; U[3] = r * W[3];
  U[4] = W[4] / G->gm1 + 0.5 * r * ((W[1] * W[1] + W[2] * W[2]) + W[3] * W[3]);
}

/* Boundary ghost state: a slip wall mirrors the normal velocity, a
 * transmissive side copies the interior state. */
static void ghost_state(int bc, const double *n, const double *W, double *Wg) {
  for (int c = 0; c < 5; ++c) Wg[c] = W[c];
  if (bc == 1) {
    double un = (W[1] * n[0] + W[2] * n[1]) + W[3] * n[2];
    for (int d = 0; d < 3; ++d) Wg[1 + d] = W[1 + d] - (2.0 * un) * n[d];
  }
}

/* minmod(a, b): 0 when the signs differ (or one is 0), else the argument of
 * smaller magnitude. */
static double minmod(double a, double b) {
  if (a > 0.0 && b > 0.0) return a < b ? a : b;
  if (a < 0.0 && b < 0.0) return a > b ? a : b;
  return 0.0;
}

/* MUSCL reconstruction of both face states (primitives):
 *   W_L = W_i + 1/2 minmod(2 g_i.r - dW, dW)
 *   W_R = W_j - 1/2 minmod(2 g_j.r - dW, dW),  dW = W_j - W_i, r = x_j - x_i */
static void muscl_pair(const double *Wi, const double *Wj, const double *gi, const double *gj,
                       const double *r, double *WL, double *WR) {
  for (int c = 0; c < 5; ++c) {
    double dW = Wj[c] - Wi[c];
    double gir = (gi[3 * c] * r[0] + gi[3 * c + 1] * r[1]) + gi[3 * c + 2] * r[2];
    double gjr = (gj[3 * c] * r[0] + gj[3 * c + 1] * r[1]) + gj[3 * c + 2] * r[2];
    WL[c] = Wi[c] + 0.5 * minmod(2.0 * gir - dW, dW);
    WR[c] = Wj[c] - 0.5 * minmod(2.0 * gjr - dW, dW);
  }
}

/* ============================================================== mesh === */
typedef struct {
  int64_t k[3];
  int64_t tet;
  int j;
} facerec;

static int cmp_facerec(const void *a, const void *b) {
  const facerec *x = (const facerec *)a, *y = (const facerec *)b;
  for (int i = 0; i < 3; ++i) {
    if (x->k[i] < y->k[i]) return -1;
    if (x->k[i] > y->k[i]) return 1;
  }
  if (x->tet < y->tet) return -1;
  if (x->tet > y->tet) return 1;
  return 0;
}

static void sort3(int64_t *k) {
  int64_t t;
  if (k[0] > k[1]) { t = k[0]; k[0] = k[1]; k[1] = t; }
  if (k[1] > k[2]) { t = k[1]; k[1] = k[2]; k[2] = t; }
  if (k[0] > k[1]) { t = k[0]; k[0] = k[1]; k[1] = t; }
}

static void vsub(const double *a, const double *b, double *o) {
  o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2];
}
static void vcross(const double *a, const double *b, double *o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
static double vdot(const double *a, const double *b) { return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2]; }

void orc_free(orc *o) {
  if (!o) return;
  void *p[] = {o->vol, o->xc, o->cface, o->csgn, o->lsw, o->fown, o->fnb, o->fbc, o->farea,
               o->fnrm, o->fr, o->U, o->Us, o->W, o->G, o->F1A, o->ACC, o->BND, o->dt,
               o->lev, o->flev, o->mark};
  for (size_t i = 0; i < sizeof p / sizeof p[0]; ++i) free(p[i]);
  free(o);
}

int orc_create(const double *xyz, int64_t n_nodes, const int64_t *tets, int64_t n_tets,
               const int8_t *face_bc, double gamma, double cfl, double newton_tol,
               int max_levels, int newton_max_iter, orc **out) {
  *out = NULL;
  if (n_tets <= 0 || n_nodes <= 0 || max_levels < 1 || max_levels > ORC_MAXL || !(gamma > 1.0) ||
      !(cfl > 0.0) || !(newton_tol > 0.0) || newton_max_iter < 1) {
    set_msg("orc_create: invalid argument");
    return ORC_EINVAL;
  }
  orc *o = (orc *)calloc(1, sizeof(orc));
  o->gas.g = gamma;
  o->gas.gm1 = gamma - 1.0;
  o->gas.gp1 = gamma + 1.0;
  o->gas.tol = newton_tol;
  o->gas.maxit = newton_max_iter;
  o->cfl = cfl;
  o->L = max_levels;
  o->theta = max_levels - 1;
  int64_t nc = n_tets;
  o->nc = nc;
  o->vol = malloc(sizeof(double) * nc);
  o->xc = malloc(sizeof(double) * 3 * nc);
  o->cface = malloc(sizeof(int64_t) * 4 * nc);
  o->csgn = malloc(4 * nc);
  o->lsw = malloc(sizeof(double) * 12 * nc);

  /* cell volume and centroid */
  for (int64_t i = 0; i < nc; ++i) {
    const double *x[4];
    for (int v = 0; v < 4; ++v) {
      int64_t nd = tets[4 * i + v];
      if (nd < 0 || nd >= n_nodes) {
        set_msg("orc_create: node index out of range");
        orc_free(o);
        return ORC_EMESH;
      }
      x[v] = xyz + 3 * nd;
    }
    double e1[3], e2[3], e3[3], c[3];
    vsub(x[1], x[0], e1);
    vsub(x[2], x[0], e2);
    vsub(x[3], x[0], e3);
    vcross(e1, e2, c);
    double V = vdot(c, e3) / 6.0;
    if (!(V > 0.0)) {
      set_msg("orc_create: non-positive tet volume");
      orc_free(o);
      return ORC_EMESH;
    }
    o->vol[i] = V;
    for (int d = 0; d < 3; ++d) o->xc[3 * i + d] = (((x[0][d] + x[1][d]) + x[2][d]) + x[3][d]) * 0.25;
  }

  /* faces: sort the 4 nc (sorted node triple) records, pair equal keys */
  facerec *rec = malloc(sizeof(facerec) * 4 * nc);
  for (int64_t i = 0; i < nc; ++i)
    for (int j = 0; j < 4; ++j) {
      facerec *r = &rec[4 * i + j];
      int m = 0;
      for (int v = 0; v < 4; ++v)
        if (v != j) r->k[m++] = tets[4 * i + v];
      sort3(r->k);
      r->tet = i;
      r->j = j;
    }
  qsort(rec, 4 * nc, sizeof(facerec), cmp_facerec);
  int64_t nf = 0;
  for (int64_t a = 0; a < 4 * nc;) {
    int64_t b = a + 1;
    while (b < 4 * nc && memcmp(rec[b].k, rec[a].k, sizeof rec[a].k) == 0) ++b;
    if (b - a > 2) {
      set_msg("orc_create: non-manifold face (shared by more than two tets)");
      free(rec);
      orc_free(o);
      return ORC_EMESH;
    }
    ++nf;
    a = b;
  }
  o->nf = nf;
  o->fown = malloc(sizeof(int64_t) * nf);
  o->fnb = malloc(sizeof(int64_t) * nf);
  o->fbc = malloc(nf);
  o->farea = malloc(sizeof(double) * nf);
  o->fnrm = malloc(sizeof(double) * 3 * nf);
  o->fr = malloc(sizeof(double) * 3 * nf);
  int64_t f = 0;
  for (int64_t a = 0; a < 4 * nc;) {
    int64_t b = a + 1;
    while (b < 4 * nc && memcmp(rec[b].k, rec[a].k, sizeof rec[a].k) == 0) ++b;
    const facerec *ow = &rec[a]; /* lower tet index owns the face */
    int8_t bco = face_bc[4 * ow->tet + ow->j];
    o->fown[f] = ow->tet;
    o->cface[4 * ow->tet + ow->j] = f;
    o->csgn[4 * ow->tet + ow->j] = 1;
    if (b - a == 2) {
      const facerec *nb = &rec[a + 1];
      if (bco != 0 || face_bc[4 * nb->tet + nb->j] != 0) {
        set_msg("orc_create: interior face carries a boundary tag");
        free(rec);
        orc_free(o);
        return ORC_EMESH;
      }
      o->fnb[f] = nb->tet;
      o->fbc[f] = 0;
      o->cface[4 * nb->tet + nb->j] = f;
      o->csgn[4 * nb->tet + nb->j] = -1;
    } else {
      if (bco != 1 && bco != 2) {
        set_msg("orc_create: boundary face without a wall/transmissive tag");
        free(rec);
        orc_free(o);
        return ORC_EMESH;
      }
      o->fnb[f] = -1;
      o->fbc[f] = bco;
    }
    /* area vector of the owner's local face j (nodes in ascending local
     * order), oriented away from the opposite node */
    const int64_t *tv = tets + 4 * ow->tet;
    const double *q[3];
    int m = 0;
    for (int v = 0; v < 4; ++v)
      if (v != ow->j) q[m++] = xyz + 3 * tv[v];
    const double *xo = xyz + 3 * tv[ow->j];
    double e1[3], e2[3], av[3], to[3];
    vsub(q[1], q[0], e1);
    vsub(q[2], q[0], e2);
    vcross(e1, e2, av);
    for (int d = 0; d < 3; ++d) av[d] *= 0.5;
    vsub(xo, q[0], to);
    if (vdot(av, to) > 0.0)
      for (int d = 0; d < 3; ++d) av[d] = -av[d];
    double A = sqrt(vdot(av, av));
    o->farea[f] = A;
    for (int d = 0; d < 3; ++d) o->fnrm[3 * f + d] = av[d] / A;
    double xf[3];
    for (int d = 0; d < 3; ++d) xf[d] = ((q[0][d] + q[1][d]) + q[2][d]) / 3.0;
    const double *xl = o->xc + 3 * ow->tet;
    if (o->fnb[f] >= 0) {
      const double *xr = o->xc + 3 * o->fnb[f];
      for (int d = 0; d < 3; ++d) o->fr[3 * f + d] = xr[d] - xl[d];
    } else { /* ghost centroid: mirror of the cell centroid in the face plane */
      double dl[3];
      vsub(xf, xl, dl);
      double s = 2.0 * vdot(dl, o->fnrm + 3 * f);
      for (int d = 0; d < 3; ++d) o->fr[3 * f + d] = s * o->fnrm[3 * f + d];
    }
    ++f;
    a = b;
  }
  free(rec);

  /* least-squares weights: w_j = M^-1 r_j, M = sum_j r_j r_j^T */
  for (int64_t i = 0; i < nc; ++i) {
    double r[4][3];
    for (int j = 0; j < 4; ++j) {
      int64_t fj = o->cface[4 * i + j];
      double s = o->csgn[4 * i + j] > 0 ? 1.0 : -1.0;
      for (int d = 0; d < 3; ++d) r[j][d] = s * o->fr[3 * fj + d];
    }
    double M[3][3] = {{0}};
    for (int j = 0; j < 4; ++j)
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) M[a][b] += r[j][a] * r[j][b];
    double c00 = M[1][1] * M[2][2] - M[1][2] * M[2][1];
    double c01 = M[1][2] * M[2][0] - M[1][0] * M[2][2];
    double c02 = M[1][0] * M[2][1] - M[1][1] * M[2][0];
    double det = (M[0][0] * c00 + M[0][1] * c01) + M[0][2] * c02;
    double inv[3][3];
    inv[0][0] = c00 / det;
    inv[1][0] = c01 / det;
    inv[2][0] = c02 / det;
    inv[0][1] = (M[0][2] * M[2][1] - M[0][1] * M[2][2]) / det;
    inv[1][1] = (M[0][0] * M[2][2] - M[0][2] * M[2][0]) / det;
    inv[2][1] = (M[0][1] * M[2][0] - M[0][0] * M[2][1]) / det;
    inv[0][2] = (M[0][1] * M[1][2] - M[0][2] * M[1][1]) / det;
    inv[1][2] = (M[0][2] * M[1][0] - M[0][0] * M[1][2]) / det;
    inv[2][2] = (M[0][0] * M[1][1] - M[0][1] * M[1][0]) / det;
    for (int j = 0; j < 4; ++j)
      for (int a = 0; a < 3; ++a)
        o->lsw[12 * i + 3 * j + a] = (inv[a][0] * r[j][0] + inv[a][1] * r[j][1]) + inv[a][2] * r[j][2];
  }

  o->U = calloc(5 * nc, sizeof(double));
  o->Us = calloc(5 * nc, sizeof(double));
  o->W = calloc(5 * nc, sizeof(double));
  o->G = calloc(15 * nc, sizeof(double));
  o->F1A = calloc(5 * nf, sizeof(double));
  o->ACC = calloc(5 * nf, sizeof(double));
  o->BND = calloc(5 * nf, sizeof(double));
  o->dt = calloc(nc, sizeof(double));
  o->lev = calloc(nc, 1);
  o->flev = calloc(nf, 1);
  o->mark = calloc(nc, 1);
  *out = o;
  return ORC_OK;
}

int64_t orc_n_cells(const orc *o) { return o->nc; }
int64_t orc_n_faces(const orc *o) { return o->nf; }
double orc_time(const orc *o) { return o->t; }
double orc_dtmin(const orc *o) { return o->dtmin; }

int orc_cell_geometry(const orc *o, double *vol, double *xc_soa) {
  for (int64_t i = 0; i < o->nc; ++i) {
    vol[i] = o->vol[i];
    for (int d = 0; d < 3; ++d) xc_soa[d * o->nc + i] = o->xc[3 * i + d];
  }
  return ORC_OK;
}

int orc_face_data(const orc *o, int64_t *own, int64_t *nb, int8_t *bc, double *area,
                  double *nrm_soa) {
  for (int64_t f = 0; f < o->nf; ++f) {
    own[f] = o->fown[f];
    nb[f] = o->fnb[f];
    bc[f] = o->fbc[f];
    area[f] = o->farea[f];
    for (int d = 0; d < 3; ++d) nrm_soa[d * o->nf + f] = o->fnrm[3 * f + d];
  }
  return ORC_OK;
}

/* ============================================================= state === */
static int check_state(const orc *o, const double *U, int64_t i) {
  double W[5];
  cons_to_prim(&o->gas, U + 5 * i, W);
  return (W[0] > 0.0 && W[4] > 0.0 && isfinite(W[0]) && isfinite(W[4]) && isfinite(W[1]) &&
          isfinite(W[2]) && isfinite(W[3]));
}

int orc_set_prim(orc *o, const double *prim_soa) {
  for (int64_t i = 0; i < o->nc; ++i) {
    double W[5];
    for (int c = 0; c < 5; ++c) W[c] = prim_soa[c * o->nc + i];
    if (!(W[0] > 0.0 && W[4] > 0.0)) {
      set_msg("orc_set_prim: non-positive density or pressure");
      return ORC_ENONPHYS;
    }
    prim_to_cons(&o->gas, W, o->U + 5 * i);
  }
  memcpy(o->Us, o->U, sizeof(double) * 5 * o->nc);
  memset(o->ACC, 0, sizeof(double) * 5 * o->nf);
  memset(o->BND, 0, sizeof(double) * 5 * o->nf);
  o->have_levels = 0;
  o->next_phase = 0;
  return ORC_OK;
}

int orc_set_cons(orc *o, const double *cons_soa) {
  for (int64_t i = 0; i < o->nc; ++i)
    for (int c = 0; c < 5; ++c) o->U[5 * i + c] = cons_soa[c * o->nc + i];
  memcpy(o->Us, o->U, sizeof(double) * 5 * o->nc);
  memset(o->ACC, 0, sizeof(double) * 5 * o->nf);
  memset(o->BND, 0, sizeof(double) * 5 * o->nf);
  o->have_levels = 0;
  o->next_phase = 0;
  return ORC_OK;
}

int orc_get_cons(const orc *o, double *cons_soa) {
  for (int64_t i = 0; i < o->nc; ++i)
    for (int c = 0; c < 5; ++c) cons_soa[c * o->nc + i] = o->U[5 * i + c];
  return ORC_OK;
}

int orc_get_pred(const orc *o, double *cons_soa) {
  for (int64_t i = 0; i < o->nc; ++i)
    for (int c = 0; c < 5; ++c) cons_soa[c * o->nc + i] = o->Us[5 * i + c];
  return ORC_OK;
}

void orc_set_time(orc *o, double t) { o->t = t; }

/* ========================================================== levels ===== */
/* Local explicit step: dt_i = 2 CFL V_i / sum_f A_f (|u_i . n_f| + c_i),
 * evaluated with rho_i multiplied through numerator and denominator:
 *   dt_i = 2 CFL V_i rho_i / sum_f A_f (|m_i . n_f| + rho_i c_i),
 * m = rho u, rho c = sqrt(gamma p rho), p = (gamma-1)(E - (|m|^2/2)/rho). */
static double local_dt(const orc *o, int64_t i) {
  const double *U = o->U + 5 * i;
  double r = U[0];
  double mm = (U[1] * U[1] + U[2] * U[2]) + U[3] * U[3];
  double p = o->gas.gm1 * (U[4] - (0.5 * mm) / r);
  double rc = sqrt((o->gas.g * p) * r);
  double S = 0.0;
  for (int j = 0; j < 4; ++j) {
    int64_t f = o->cface[4 * i + j];
    const double *n = o->fnrm + 3 * f;
    double mn = (U[1] * n[0] + U[2] * n[1]) + U[3] * n[2];
    S = S + o->farea[f] * (fabs(mn) + rc);
  }
  return (((2.0 * o->cfl) * o->vol[i]) * r) / S;
}

/* Alg. 2, time steps and levels: Delta t = min_i dt_i; level k_i = the largest k in
 * [0, L-1] with 2^k Delta t <= dt_i; then lower levels until every pair of
 * neighbours differs by at most one (repeated until nothing changes). */
int orc_assign_levels(orc *o, double *dtmin_out, int8_t *levels_out, int32_t *counts_out) {
  if (o->have_levels && o->next_phase > 0) {
    set_msg("orc_assign_levels: a cycle is in progress");
    return ORC_EINVAL;
  }
  for (int64_t i = 0; i < o->nc; ++i)
    if (!check_state(o, o->U, i)) {
      set_msg("orc_assign_levels: non-physical state");
      return ORC_ENONPHYS;
    }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < o->nc; ++i) o->dt[i] = local_dt(o, i);
  double m = o->dt[0];
  for (int64_t i = 1; i < o->nc; ++i)
    if (o->dt[i] < m) m = o->dt[i];
  o->dtmin = m;
  for (int64_t i = 0; i < o->nc; ++i) {
    int k = 0;
    while (k + 1 < o->L && ldexp(m, k + 1) <= o->dt[i]) ++k;
    o->lev[i] = (int8_t)k;
  }
  int changed = 1;
  while (changed) {
    changed = 0;
    for (int64_t i = 0; i < o->nc; ++i)
      for (int j = 0; j < 4; ++j) {
        int64_t f = o->cface[4 * i + j];
        int64_t nb = o->csgn[4 * i + j] > 0 ? o->fnb[f] : o->fown[f];
        if (nb < 0) continue;
        if (o->lev[i] > o->lev[nb] + 1) {
          o->lev[i] = (int8_t)(o->lev[nb] + 1);
          changed = 1;
        }
      }
  }
  for (int64_t f = 0; f < o->nf; ++f) {
    int8_t a = o->lev[o->fown[f]];
    int8_t b = o->fnb[f] >= 0 ? o->lev[o->fnb[f]] : a;
    o->flev[f] = a < b ? a : b;
  }
  for (int k = 0; k < ORC_MAXL; ++k) {
    o->tn[k] = 0;
    o->pred[k] = 0;
  }
  memcpy(o->Us, o->U, sizeof(double) * 5 * o->nc);
  o->have_levels = 1;
  o->next_phase = 0;
  if (dtmin_out) *dtmin_out = m;
  if (levels_out) memcpy(levels_out, o->lev, o->nc);
  if (counts_out) {
    for (int k = 0; k < o->L; ++k) counts_out[k] = 0;
    for (int64_t i = 0; i < o->nc; ++i) counts_out[o->lev[i]]++;
  }
  return ORC_OK;
}

int orc_get_levels(const orc *o, int8_t *levels_out) {
  memcpy(levels_out, o->lev, o->nc);
  return ORC_OK;
}

/* ===================================================== time-level logic */
/* The state of cell i at time T (Delta t units from the cycle start), by
 * linear interpolation between U^n (at tn) and U* (at tn + 2^k). */
static void state_at(const orc *o, int64_t i, int64_t T, double *Ui) {
  int k = o->lev[i];
  int64_t num = T - o->tn[k];
  const double *a = o->U + 5 * i, *b = o->Us + 5 * i;
  if (num == 0) {
    for (int c = 0; c < 5; ++c) Ui[c] = a[c];
  } else if (num == ((int64_t)1 << k)) {
    for (int c = 0; c < 5; ++c) Ui[c] = b[c];
  } else {
    double w = ldexp((double)num, -k);
    for (int c = 0; c < 5; ++c) Ui[c] = a[c] + w * (b[c] - a[c]);
  }
}

/* states of every level valid at T? (tn_k <= T <= tn_k + 2^k, and U* valid
 * when T > tn_k) */
static int states_valid(const orc *o, int64_t T, const int *present) {
  for (int k = 0; k < o->L; ++k) {
    if (!present[k]) continue;
    int64_t d = T - o->tn[k];
    if (d < 0 || d > ((int64_t)1 << k)) return 0;
    if (d > 0 && !o->pred[k]) return 0;
  }
  return 1;
}

static void compute_W(orc *o, int64_t T) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < o->nc; ++i) {
    double Ui[5];
    state_at(o, i, T, Ui);
    cons_to_prim(&o->gas, Ui, o->W + 5 * i);
  }
}

/* least-squares gradient of the five primitives of cell i from its four face
 * neighbours (ghost states on boundary faces) */
static void gradient_cell(orc *o, int64_t i) {
  double *g = o->G + 15 * i;
  const double *Wi = o->W + 5 * i;
  for (int q = 0; q < 15; ++q) g[q] = 0.0;
  for (int j = 0; j < 4; ++j) {
    int64_t f = o->cface[4 * i + j];
    int64_t nb = o->csgn[4 * i + j] > 0 ? o->fnb[f] : o->fown[f];
    double Wn[5];
    if (nb >= 0) {
      for (int c = 0; c < 5; ++c) Wn[c] = o->W[5 * nb + c];
    } else {
      ghost_state(o->fbc[f], o->fnrm + 3 * f, Wi, Wn);
    }
    const double *w = o->lsw + 12 * i + 3 * j;
    for (int c = 0; c < 5; ++c) {
      double d = Wn[c] - Wi[c];
      for (int a = 0; a < 3; ++a) g[3 * c + a] += w[a] * d;
    }
  }
}

static void compute_gradients_marked(orc *o) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < o->nc; ++i)
    if (o->mark[i]) gradient_cell(o, i);
}

/* Boundary fluxes (per unit area), equal to the Godunov flux against the
 * ghost state but written so that the invariants hold exactly:
 *  - slip wall: the Riemann problem (rho, u_n, p | rho, -u_n, p) has u* = 0,
 *    so the flux is (0, p* n, 0): no mass or energy crosses a wall;
 *  - transmissive: identical states, so the flux is the physical flux of W_L. */
static int boundary_flux(const gas_t *G, int bc, const double *WL, const double *n, double *F,
                         int *iters) {
  double un = (WL[1] * n[0] + WL[2] * n[1]) + WL[3] * n[2];
  if (bc == 1) {
    double ps, us;
    int rc = riemann_star(G, WL[0], un, WL[4], WL[0], -un, WL[4], &ps, &us, iters);
    if (rc) return rc;
    F[0] = 0.0;
    for (int d = 0; d < 3; ++d) F[1 + d] = ps * n[d];
    F[4] = 0.0;
    return ORC_OK;
  }
  *iters = 0;
  double r = WL[0], p = WL[4];
  double E = p / G->gm1 + 0.5 * r * ((WL[1] * WL[1] + WL[2] * WL[2]) + WL[3] * WL[3]);
  double mass = r * un;
  F[0] = mass;
  for (int d = 0; d < 3; ++d) F[1 + d] = mass * WL[1 + d] + p * n[d];
  F[4] = un * (E + p);
  return ORC_OK;
}

/* flux F A through face f from the current W and G */
static int face_flux_A(const orc *o, int64_t f, double *FA, int *iters) {
  int64_t L = o->fown[f], R = o->fnb[f];
  const double *n = o->fnrm + 3 * f;
  const double *r = o->fr + 3 * f;
  double WL[5], WR[5], F[5];
  int rc;
  if (R >= 0) {
    muscl_pair(o->W + 5 * L, o->W + 5 * R, o->G + 15 * L, o->G + 15 * R, r, WL, WR);
    rc = godunov_flux(&o->gas, WL, WR, n, F, iters);
  } else {
    /* W_L is reconstructed towards the ghost cell (mirror image of the cell
     * in the face plane); the ghost's own reconstruction is not needed */
    double Wg[5];
    ghost_state(o->fbc[f], n, o->W + 5 * L, Wg);
    muscl_pair(o->W + 5 * L, Wg, o->G + 15 * L, o->G + 15 * L, r, WL, WR);
    rc = boundary_flux(&o->gas, o->fbc[f], WL, n, F, iters);
  }
  if (rc) return rc;
  for (int c = 0; c < 5; ++c) FA[c] = F[c] * o->farea[f];
  return ORC_OK;
}

/* The phases of one cycle: for s = 1..2^theta, B(s) then E(s,0..e(s)). */
typedef struct {
  int kind; /* 0 begin, 1 end */
  int level; /* begin: tau(s); end: the level that completes */
  int64_t T; /* phase time, Delta t units from the cycle start */
} phase_t;

static int n_phases(int theta) { return 3 * (1 << theta) - 1; }

static phase_t phase_at(int theta, int idx) {
  phase_t ph = {0, 0, 0};
  int nsub = 1 << theta;
  for (int s = 1; s <= nsub; ++s) {
    /* Alg. 2, subiteration s: tau = largest tmp <= theta with (s-1) mod 2^tmp == 0 */
    int tau = 0;
    for (int tmp = 1; tmp <= theta; ++tmp)
      if (((s - 1) % (1 << tmp)) == 0) tau = tmp;
    if (idx == 0) {
      ph.kind = 0; ph.level = tau; ph.T = s - 1;
      return ph;
    }
    --idx;
    for (int k = 0; k <= theta && (s % (1 << k)) == 0; ++k) {
      if (idx == 0) {
        ph.kind = 1; ph.level = k; ph.T = s;
        return ph;
      }
      --idx;
    }
  }
  return ph;
}

/* Order 1, the order of Alg. 2's subiteration loop (Sec. 2.2).  Subiteration
 * s with tau = tau(s) and T0 = s - 1:
 *   - if s > 1, commit(tau, T0): the levels <= tau, whose steps end at T0,
 *     take their end states with the intensive correction of Alg. 2 -- the
 *     provisional integral of each face to a finer neighbour is replaced by
 *     the integral the finer cells accumulated over the step;
 *   - begin(tau, T0), the predictor of the levels <= tau (as in order 0);
 *   - for tau' = tau down to 0, correct(tau', T0 + 2^tau'): the corrector of
 *     level tau' at the end of its step, computed before the finer levels
 *     have advanced: finer neighbours enter its gradients extrapolated
 *     linearly in time from U^n and U* (Alg. 2's repositioning), and each
 *     face to a finer neighbour enters with the provisional integral
 *     dt_k F1 A; the result is the level's provisional end state.
 * After the last subiteration, commit(theta, 2^theta) -- the extra pass of
 * Alg. 3's loop over 2^theta + 1 subiterations.  The paper does not say
 * which provisional interface flux its coarse corrector uses; the predictor
 * flux F1 is the reading taken here.  Kinds: 0 begin, 2 correct, 3 commit. */
static int n_phases_paper(int theta) { return 4 * (1 << theta) - 1; }

static phase_t phase_at_paper(int theta, int idx) {
  phase_t ph = {3, theta, (int64_t)1 << theta};
  int nsub = 1 << theta;
  for (int s = 1; s <= nsub; ++s) {
    int tau = 0;
    for (int tmp = 1; tmp <= theta; ++tmp)
      if (((s - 1) % (1 << tmp)) == 0) tau = tmp;
    if (s > 1) {
      if (idx == 0) {
        ph.kind = 3; ph.level = tau; ph.T = s - 1;
        return ph;
      }
      --idx;
    }
    if (idx == 0) {
      ph.kind = 0; ph.level = tau; ph.T = s - 1;
      return ph;
    }
    --idx;
    for (int k = tau; k >= 0; --k) {
      if (idx == 0) {
        ph.kind = 2; ph.level = k; ph.T = (s - 1) + ((int64_t)1 << k);
        return ph;
      }
      --idx;
    }
  }
  return ph; /* the final commit */
}

/* Begin(s): every level <= tau starts a step at T: fluxes F1 on every face
 * of face-level <= tau, then the predictor U* = U^n + dt_k R(U^n). */
static int phase_begin(orc *o, int tau, int64_t T) {
  compute_W(o, T);
  memset(o->mark, 0, o->nc);
  for (int64_t f = 0; f < o->nf; ++f)
    if (o->flev[f] <= tau) {
      o->mark[o->fown[f]] = 1;
      if (o->fnb[f] >= 0) o->mark[o->fnb[f]] = 1;
    }
  compute_gradients_marked(o);
  int err = 0;
  int64_t iters = 0, calls = 0;
#pragma omp parallel for schedule(static) reduction(| : err) reduction(+ : iters, calls)
  for (int64_t f = 0; f < o->nf; ++f)
    if (o->flev[f] <= tau) {
      int it = 0;
      if (face_flux_A(o, f, o->F1A + 5 * f, &it)) err |= 1;
      iters += it;
      calls += 1;
    }
  o->newton_iters += iters;
  o->riemann_calls += calls;
  for (int k = 0; k <= tau; ++k) {
    int64_t cnt = 0;
    for (int64_t f = 0; f < o->nf; ++f) cnt += (o->flev[f] == k);
    o->n_faceevals[k] += cnt;
  }
  if (err) {
    set_msg("Riemann solver failed (vacuum or no convergence)");
    return ORC_ERIEMANN;
  }
#pragma omp parallel for schedule(static) reduction(| : err)
  for (int64_t i = 0; i < o->nc; ++i) {
    int k = o->lev[i];
    if (k > tau) continue;
    double S[5] = {0, 0, 0, 0, 0};
    for (int j = 0; j < 4; ++j) {
      int64_t f = o->cface[4 * i + j];
      double s = o->csgn[4 * i + j];
      for (int c = 0; c < 5; ++c) S[c] += s * o->F1A[5 * f + c];
    }
    double dtk = ldexp(o->dtmin, k);
    for (int c = 0; c < 5; ++c) {
      double R = -S[c] / o->vol[i];
      o->Us[5 * i + c] = o->U[5 * i + c] + dtk * R;
    }
    if (!check_state(o, o->Us, i)) err |= 1;
  }
  for (int k = 0; k <= tau; ++k) o->pred[k] = 1;
  if (err) {
    set_msg("non-physical predicted state");
    return ORC_ENONPHYS;
  }
  return ORC_OK;
}

/* End of the level-k step at T: fluxes F2 on face-level-k faces,
 * Phi = dt_k (F1 + F2)/2 A, accumulation on level interfaces, then the
 * corrector U^{n+1} = U^n - sum sigma Phi / V (faces to finer neighbours
 * contribute their accumulated fine-side integral, which is then reset). */
static int phase_end(orc *o, int k, int64_t T) {
  compute_W(o, T);
  memset(o->mark, 0, o->nc);
  for (int64_t f = 0; f < o->nf; ++f)
    if (o->flev[f] == k) {
      o->mark[o->fown[f]] = 1;
      if (o->fnb[f] >= 0) o->mark[o->fnb[f]] = 1;
    }
  compute_gradients_marked(o);
  double dtk = ldexp(o->dtmin, k);
  int err = 0;
  int64_t iters = 0, calls = 0, cnt = 0;
#pragma omp parallel for schedule(static) reduction(| : err) reduction(+ : iters, calls, cnt)
  for (int64_t f = 0; f < o->nf; ++f)
    if (o->flev[f] == k) {
      double F2A[5];
      int it = 0;
      if (face_flux_A(o, f, F2A, &it)) {
        err |= 1;
        continue;
      }
      iters += it;
      calls += 1;
      cnt += 1;
      int interface = o->fnb[f] >= 0 && o->lev[o->fown[f]] != o->lev[o->fnb[f]];
      for (int c = 0; c < 5; ++c) {
        double phi = dtk * (0.5 * (o->F1A[5 * f + c] + F2A[c]));
        o->F1A[5 * f + c] = phi;
        if (interface) o->ACC[5 * f + c] += phi;
        if (o->fnb[f] < 0) o->BND[5 * f + c] += phi;
      }
    }
  o->newton_iters += iters;
  o->riemann_calls += calls;
  o->n_faceevals[k] += cnt;
  if (err) {
    set_msg("Riemann solver failed (vacuum or no convergence)");
    return ORC_ERIEMANN;
  }
  int64_t upd = 0;
#pragma omp parallel for schedule(static) reduction(| : err) reduction(+ : upd)
  for (int64_t i = 0; i < o->nc; ++i) {
    if (o->lev[i] != k) continue;
    double S[5] = {0, 0, 0, 0, 0};
    for (int j = 0; j < 4; ++j) {
      int64_t f = o->cface[4 * i + j];
      double s = o->csgn[4 * i + j];
      const double *phi = o->flev[f] == k ? o->F1A + 5 * f : o->ACC + 5 * f;
      for (int c = 0; c < 5; ++c) S[c] += s * phi[c];
    }
    for (int j = 0; j < 4; ++j) {
      int64_t f = o->cface[4 * i + j];
      if (o->flev[f] < k)
        for (int c = 0; c < 5; ++c) o->ACC[5 * f + c] = 0.0;
    }
    for (int c = 0; c < 5; ++c) o->U[5 * i + c] = o->U[5 * i + c] - S[c] / o->vol[i];
    if (!check_state(o, o->U, i)) err |= 1;
    upd += 1;
  }
  o->n_updates[k] += upd;
  o->tn[k] = T;
  o->pred[k] = 0;
  if (err) {
    set_msg("non-physical corrected state");
    return ORC_ENONPHYS;
  }
  return ORC_OK;
}

/* Order 1: the corrector of level k computed at the end T of its step
 * (see phase_at_paper).  Fluxes F2 and Phi = dt_k (F1 + F2)/2 A on the
 * face-level-k faces exactly as in phase_end; the cells of level k get the
 * provisional end state U^n - sum sigma phi / V in Us, where phi is Phi on
 * their own-level faces (and faces to coarser neighbours) and dt_k F1 A on
 * faces to finer neighbours, whose accumulator starts at minus that value. */
static int phase_correct(orc *o, int k, int64_t T) {
  compute_W(o, T);
  memset(o->mark, 0, o->nc);
  for (int64_t f = 0; f < o->nf; ++f)
    if (o->flev[f] == k) {
      o->mark[o->fown[f]] = 1;
      if (o->fnb[f] >= 0) o->mark[o->fnb[f]] = 1;
    }
  compute_gradients_marked(o);
  double dtk = ldexp(o->dtmin, k);
  int err = 0;
  int64_t iters = 0, calls = 0, cnt = 0;
#pragma omp parallel for schedule(static) reduction(| : err) reduction(+ : iters, calls, cnt)
  for (int64_t f = 0; f < o->nf; ++f)
    if (o->flev[f] == k) {
      double F2A[5];
      int it = 0;
      if (face_flux_A(o, f, F2A, &it)) {
        err |= 1;
        continue;
      }
      iters += it;
      calls += 1;
      cnt += 1;
      int interface = o->fnb[f] >= 0 && o->lev[o->fown[f]] != o->lev[o->fnb[f]];
      for (int c = 0; c < 5; ++c) {
        double phi = dtk * (0.5 * (o->F1A[5 * f + c] + F2A[c]));
        o->F1A[5 * f + c] = phi;
        if (interface) o->ACC[5 * f + c] += phi;
        if (o->fnb[f] < 0) o->BND[5 * f + c] += phi;
      }
    }
  o->newton_iters += iters;
  o->riemann_calls += calls;
  o->n_faceevals[k] += cnt;
  if (err) {
    set_msg("Riemann solver failed (vacuum or no convergence)");
    return ORC_ERIEMANN;
  }
  int64_t upd = 0;
#pragma omp parallel for schedule(static) reduction(| : err) reduction(+ : upd)
  for (int64_t i = 0; i < o->nc; ++i) {
    if (o->lev[i] != k) continue;
    double S[5] = {0, 0, 0, 0, 0};
    for (int j = 0; j < 4; ++j) {
      int64_t f = o->cface[4 * i + j];
      double s = o->csgn[4 * i + j];
      if (o->flev[f] == k) {
        for (int c = 0; c < 5; ++c) S[c] += s * o->F1A[5 * f + c];
      } else { /* a finer neighbour: provisional integral from the predictor flux */
        for (int c = 0; c < 5; ++c) {
          double prov = dtk * o->F1A[5 * f + c];
          S[c] += s * prov;
          o->ACC[5 * f + c] -= prov;
        }
      }
    }
    for (int c = 0; c < 5; ++c) o->Us[5 * i + c] = o->U[5 * i + c] - S[c] / o->vol[i];
    if (!check_state(o, o->Us, i)) err |= 1;
    upd += 1;
  }
  o->n_updates[k] += upd;
  if (err) {
    set_msg("non-physical corrected state");
    return ORC_ENONPHYS;
  }
  return ORC_OK;
}

/* Order 1: the levels <= tau end their steps at T (Alg. 2's intensive
 * correction): U^{n+1} = Us - sum sigma ACC / V over the faces to finer
 * neighbours (ACC = the finer side's integral minus the provisional one),
 * which are then reset; a cell without finer neighbours takes Us as it is. */
static int phase_commit(orc *o, int tau, int64_t T) {
  int err = 0;
#pragma omp parallel for schedule(static) reduction(| : err)
  for (int64_t i = 0; i < o->nc; ++i) {
    int k = o->lev[i];
    if (k > tau) continue;
    int any = 0;
    double S[5] = {0, 0, 0, 0, 0};
    for (int j = 0; j < 4; ++j) {
      int64_t f = o->cface[4 * i + j];
      if (o->flev[f] >= k) continue;
      double s = o->csgn[4 * i + j];
      for (int c = 0; c < 5; ++c) S[c] += s * o->ACC[5 * f + c];
      any = 1;
    }
    for (int j = 0; j < 4; ++j) {
      int64_t f = o->cface[4 * i + j];
      if (o->flev[f] < k)
        for (int c = 0; c < 5; ++c) o->ACC[5 * f + c] = 0.0;
    }
    for (int c = 0; c < 5; ++c)
      o->U[5 * i + c] = any ? o->Us[5 * i + c] - S[c] / o->vol[i] : o->Us[5 * i + c];
    if (!check_state(o, o->U, i)) err |= 1;
  }
  for (int k = 0; k <= tau; ++k) {
    o->tn[k] = T;
    o->pred[k] = 0;
  }
  if (err) {
    set_msg("non-physical corrected state");
    return ORC_ENONPHYS;
  }
  return ORC_OK;
}

static int phases_per_cycle(const orc *o) {
  return o->order == 1 ? n_phases_paper(o->theta) : n_phases(o->theta);
}

int orc_set_order(orc *o, int order) {
  if ((order != 0 && order != 1) || (o->have_levels && o->next_phase > 0)) {
    set_msg("orc_set_order: order 0 or 1, between cycles");
    return ORC_EINVAL;
  }
  o->order = order;
  return ORC_OK;
}

/* run n phases of the current cycle (levels must be assigned) */
int orc_run_phases(orc *o, int n) {
  if (!o->have_levels) {
    set_msg("orc_run_phases: levels not assigned");
    return ORC_EINVAL;
  }
  int total = phases_per_cycle(o);
  for (int q = 0; q < n; ++q) {
    if (o->next_phase >= total) {
      set_msg("orc_run_phases: past the end of the cycle");
      return ORC_EINVAL;
    }
    phase_t ph = o->order == 1 ? phase_at_paper(o->theta, o->next_phase) : phase_at(o->theta, o->next_phase);
    int rc = ph.kind == 0   ? phase_begin(o, ph.level, ph.T)
             : ph.kind == 1 ? phase_end(o, ph.level, ph.T)
             : ph.kind == 2 ? phase_correct(o, ph.level, ph.T)
                            : phase_commit(o, ph.level, ph.T);
    if (rc) return rc;
    o->next_phase++;
    if (o->next_phase == total) { /* cycle complete */
      o->t += ldexp(o->dtmin, o->theta);
      o->have_levels = 0;
      o->next_phase = 0;
    }
  }
  return ORC_OK;
}

int orc_phases_per_cycle(const orc *o) { return phases_per_cycle(o); }

int orc_advance(orc *o, int n_cycles, double *t_out) {
  for (int c = 0; c < n_cycles; ++c) {
    int rc;
    if (!o->have_levels) {
      rc = orc_assign_levels(o, NULL, NULL, NULL);
      if (rc) return rc;
    }
    rc = orc_run_phases(o, phases_per_cycle(o) - o->next_phase);
    if (rc) return rc;
  }
  if (t_out) *t_out = o->t;
  return ORC_OK;
}

/* The residual R_i = -(1/V_i) sum_f sigma_f F_f A_f of the cells of level k
 * with every state taken at the start (stage 1) or end (stage 2) of level
 * k's current step.  Pure: changes no state.  R_soa is 5 x nc; entries of
 * other cells are set to 0. */
int orc_residual_level(orc *o, int k, int stage, double *R_soa) {
  if (!o->have_levels || k < 0 || k >= o->L || (stage != 1 && stage != 2)) {
    set_msg("orc_residual_level: invalid argument or no levels");
    return ORC_EINVAL;
  }
  int present[ORC_MAXL] = {0};
  for (int64_t i = 0; i < o->nc; ++i) present[o->lev[i]] = 1;
  int64_t T = o->tn[k] + (stage == 2 ? ((int64_t)1 << k) : 0);
  if (stage == 2 && !o->pred[k]) {
    set_msg("orc_residual_level: level has no predicted state");
    return ORC_EINVAL;
  }
  if (!states_valid(o, T, present)) {
    set_msg("orc_residual_level: states not available at that time");
    return ORC_EINVAL;
  }
  compute_W(o, T);
  memset(o->mark, 0, o->nc);
  for (int64_t f = 0; f < o->nf; ++f) {
    int a = o->lev[o->fown[f]] == k, b = o->fnb[f] >= 0 && o->lev[o->fnb[f]] == k;
    if (a || b) {
      o->mark[o->fown[f]] = 1;
      if (o->fnb[f] >= 0) o->mark[o->fnb[f]] = 1;
    }
  }
  compute_gradients_marked(o);
  double *FA = calloc(5 * o->nf, sizeof(double));
  int err = 0;
#pragma omp parallel for schedule(static) reduction(| : err)
  for (int64_t f = 0; f < o->nf; ++f) {
    int a = o->lev[o->fown[f]] == k, b = o->fnb[f] >= 0 && o->lev[o->fnb[f]] == k;
    if (a || b) {
      int it;
      if (face_flux_A(o, f, FA + 5 * f, &it)) err |= 1;
    }
  }
  if (err) {
    free(FA);
    set_msg("Riemann solver failed");
    return ORC_ERIEMANN;
  }
  for (int64_t i = 0; i < o->nc; ++i) {
    for (int c = 0; c < 5; ++c) R_soa[c * o->nc + i] = 0.0;
    if (o->lev[i] != k) continue;
    double S[5] = {0, 0, 0, 0, 0};
    for (int j = 0; j < 4; ++j) {
      int64_t f = o->cface[4 * i + j];
      double s = o->csgn[4 * i + j];
      for (int c = 0; c < 5; ++c) S[c] += s * FA[5 * f + c];
    }
    for (int c = 0; c < 5; ++c) R_soa[c * o->nc + i] = -S[c] / o->vol[i];
  }
  free(FA);
  return ORC_OK;
}

/* One global Heun step of size dt for every cell (the classical explicit
 * method the paper compares against: every cell at the smallest step). */
int orc_global_step(orc *o, double dt) {
  compute_W(o, 0); /* tn = 0 for all levels -> U^n */
  memset(o->mark, 1, o->nc);
  /* evaluate with all levels considered level-independent */
  int8_t *save_lev = malloc(o->nc);
  memcpy(save_lev, o->lev, o->nc);
  memset(o->lev, 0, o->nc);
  int64_t save_tn0 = o->tn[0];
  o->tn[0] = 0;
  compute_W(o, 0);
  compute_gradients_marked(o);
  int err = 0;
#pragma omp parallel for schedule(static) reduction(| : err)
  for (int64_t f = 0; f < o->nf; ++f) {
    int it;
    if (face_flux_A(o, f, o->F1A + 5 * f, &it)) err |= 1;
  }
  for (int64_t i = 0; i < o->nc && !err; ++i) {
    double S[5] = {0, 0, 0, 0, 0};
    for (int j = 0; j < 4; ++j) {
      int64_t f = o->cface[4 * i + j];
      double s = o->csgn[4 * i + j];
      for (int c = 0; c < 5; ++c) S[c] += s * o->F1A[5 * f + c];
    }
    for (int c = 0; c < 5; ++c) {
      double R = -S[c] / o->vol[i];
      o->Us[5 * i + c] = o->U[5 * i + c] + dt * R;
    }
  }
  /* second stage on U* */
  double *tmp = o->U;
  o->U = o->Us;
  compute_W(o, 0);
  o->U = tmp;
  compute_gradients_marked(o);
#pragma omp parallel for schedule(static) reduction(| : err)
  for (int64_t f = 0; f < o->nf; ++f) {
    double F2A[5];
    int it;
    if (face_flux_A(o, f, F2A, &it)) {
      err |= 1;
      continue;
    }
    for (int c = 0; c < 5; ++c) {
      double phi = dt * (0.5 * (o->F1A[5 * f + c] + F2A[c]));
      o->F1A[5 * f + c] = phi;
      if (o->fnb[f] < 0) o->BND[5 * f + c] += phi;
    }
  }
  for (int64_t i = 0; i < o->nc && !err; ++i) {
    double S[5] = {0, 0, 0, 0, 0};
    for (int j = 0; j < 4; ++j) {
      int64_t f = o->cface[4 * i + j];
      double s = o->csgn[4 * i + j];
      for (int c = 0; c < 5; ++c) S[c] += s * o->F1A[5 * f + c];
    }
    for (int c = 0; c < 5; ++c) o->U[5 * i + c] = o->U[5 * i + c] - S[c] / o->vol[i];
  }
  memcpy(o->lev, save_lev, o->nc);
  free(save_lev);
  o->tn[0] = save_tn0;
  o->t += dt;
  if (err) {
    set_msg("Riemann solver failed");
    return ORC_ERIEMANN;
  }
  return ORC_OK;
}

/* sum over boundary faces of the time-integrated flux leaving the domain */
int orc_boundary_ledger(const orc *o, double *out5) {
  for (int c = 0; c < 5; ++c) out5[c] = 0.0;
  for (int64_t f = 0; f < o->nf; ++f)
    if (o->fnb[f] < 0)
      for (int c = 0; c < 5; ++c) out5[c] += o->BND[5 * f + c];
  return ORC_OK;
}

int orc_stats(const orc *o, int64_t *updates, int64_t *faceevals, int64_t *newton_iters,
              int64_t *riemann_calls) {
  for (int k = 0; k < o->L; ++k) {
    updates[k] = o->n_updates[k];
    faceevals[k] = o->n_faceevals[k];
  }
  *newton_iters = o->newton_iters;
  *riemann_calls = o->riemann_calls;
  return ORC_OK;
}

/* least-squares gradient of one scalar field q (nc) -> g (3 x nc SoA); ghost
 * values on boundary faces copy the cell's own value */
/* Least-squares gradient of a cell scalar q, through the scheme's own
 * gradient routine: q is put in every primitive slot of the scratch W and
 * gradient_cell runs on each cell; a boundary face contributes nothing
 * (its ghost copies q).  W and G are scratch that every phase recomputes. */
int orc_scalar_gradient(orc *o, const double *q, double *g_soa) {
  for (int64_t i = 0; i < o->nc; ++i)
    for (int c = 0; c < 5; ++c) o->W[5 * i + c] = q[i];
  for (int64_t i = 0; i < o->nc; ++i) {
    gradient_cell(o, i);
    for (int a = 0; a < 3; ++a) g_soa[a * o->nc + i] = o->G[15 * i + a];
  }
  return ORC_OK;
}

/* r = x_j - x_i per face (3 x nf, SoA): to the neighbour's centroid, or on a
 * boundary face to the ghost centroid (the mirror image of the cell's) */
int orc_face_offsets(const orc *o, double *r_soa) {
  for (int64_t f = 0; f < o->nf; ++f)
    for (int d = 0; d < 3; ++d) r_soa[d * o->nf + f] = o->fr[3 * f + d];
  return ORC_OK;
}

/* =================================================== standalone pieces */
int orc_riemann(double gamma, double rL, double uL, double pL, double rR, double uR, double pR,
                double tol, int maxit, double *ps, double *us, int *iters) {
  gas_t G = {gamma, gamma - 1.0, gamma + 1.0, tol, maxit};
  return riemann_star(&G, rL, uL, pL, rR, uR, pR, ps, us, iters);
}

/* exact solution of the 1D Riemann problem sampled at xi = x/t */
int orc_riemann_sample(double gamma, double rL, double uL, double pL, double rR, double uR,
                       double pR, double tol, int maxit, double xi, double *r, double *u,
                       double *p) {
  gas_t G = {gamma, gamma - 1.0, gamma + 1.0, tol, maxit};
  double ps, us;
  int it, side;
  int rc = riemann_star(&G, rL, uL, pL, rR, uR, pR, &ps, &us, &it);
  if (rc) return rc;
  riemann_sample(&G, rL, uL, pL, rR, uR, pR, ps, us, xi, r, u, p, &side);
  return ORC_OK;
}

int orc_godunov_flux(double gamma, const double *WL, const double *WR, const double *n, double tol,
                     int maxit, double *F) {
  gas_t G = {gamma, gamma - 1.0, gamma + 1.0, tol, maxit};
  int it;
  return godunov_flux(&G, WL, WR, n, F, &it);
}

int orc_boundary_flux(double gamma, int bc, const double *WL, const double *n, double tol,
                      int maxit, double *F) {
  gas_t G = {gamma, gamma - 1.0, gamma + 1.0, tol, maxit};
  int it;
  if (bc != 1 && bc != 2) return ORC_EINVAL;
  return boundary_flux(&G, bc, WL, n, F, &it);
}

int orc_ghost_state(int bc, const double *n, const double *W, double *Wg) {
  ghost_state(bc, n, W, Wg);
  return ORC_OK;
}

int orc_muscl_pair(const double *Wi, const double *Wj, const double *gi, const double *gj,
                   const double *r, double *WL, double *WR) {
  muscl_pair(Wi, Wj, gi, gj, r, WL, WR);
  return ORC_OK;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* the phase list of one cycle, for schedule checks: kind 0 = begin of the
 * levels 0..level, 1 = end of the step of `level` (order 0), 2 = corrector
 * of `level`, 3 = commit of the levels 0..level (order 1); T in Delta t
 * units from the cycle start */
int orc_phase_info(int theta, int order, int idx, int *kind, int *level, int64_t *T) {
  const int n = order == 1 ? n_phases_paper(theta) : n_phases(theta);
  if (theta < 0 || theta >= ORC_MAXL || (order != 0 && order != 1) || idx < 0 || idx >= n) return ORC_EINVAL;
  phase_t ph = order == 1 ? phase_at_paper(theta, idx) : phase_at(theta, idx);
  *kind = ph.kind;
  *level = ph.level;
  *T = ph.T;
  return ORC_OK;
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
