/*
 * FP64 CPU oracle for the generalized REV-scale lattice Boltzmann model with
 * Klinkenberg's effect (Chen, Fang, Kang, Hyman, Viswanathan, Tao,
 * arXiv:1411.7051), Sections II-III.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * reference that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or constant with the CUDA path.
 *
 * Layout: node-major ("array of structures"), f[(y*nx + x)*9 + i], FP64,
 * two arrays, push form: collide every fluid node, then stream.
 *
 * Readings of points the paper leaves open:
 *   - Eq. 15's last term is taken as -3(u.F)/(eps c^2): the only form with
 *     sum_i F_i = 0 for eps < 1 (mass conservation).
 *   - With the Forchheimer drag kept, Eq. 16b with Eq. 2 is solved as the
 *     quadratic u = v / (c0 + sqrt(c0^2 + c1|v|)) (Section III, the sentence
 *     after Eq. 17; constants derived from Eq. 2 + Eq. 16b).
 *   - eps = 0 is an impermeable node (Section III): u = 0, F = -2 m / rho
 *     (the finite limit of Eq. 16b), f_eq = w rho.
 *   - Walls are halfway bounce-back; wall rows 0 and ny-1 hold no fluid.
 *   - Pressure inlet/outlet: non-equilibrium extrapolation from the adjacent
 *     interior column (Guo, Zheng & Shi 2002), applied to the post-stream
 *     populations of columns 0 and nx-1 at every time level, t = 0 included.
 *   - Slip coefficient b = -1 for every Kn (Eq. 6); f_c(0) = 1 (limit).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- Eq. 13: D2Q9 discrete velocities, and the weights under Eq. 14 ---- */
static const int ORC_EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int ORC_EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double ORC_W[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                                1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                                1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

/* boundary kinds */
#define ORC_BC_PERIODIC 0
#define ORC_BC_PRESSURE 1 /* x only */
#define ORC_BC_WALLS 1    /* y only */

typedef struct orc_params {
  int32_t nx, ny;
  double tau;   /* dimensionless relaxation time, Eq. 12 */
  double J;     /* viscosity ratio nu_e / nu, Eq. 1b; the paper uses J = 1 */
  double Gx, Gy; /* external body force G, Eq. 2 */
  int32_t bc_x;  /* ORC_BC_PERIODIC or ORC_BC_PRESSURE */
  int32_t bc_y;  /* ORC_BC_PERIODIC or ORC_BC_WALLS */
  double rho0;   /* initial density */
  double rho_in, rho_out; /* densities imposed at x = 0 and x = nx-1 */
  int32_t forchheimer;    /* 1: keep the |u|u drag of Eq. 2; 0: Eq. 8 */
  int32_t kn_model;       /* f_c: 0 Eq. 6-7 (second order), 1 Eq. 4-5 (first order) */
  double kn_beta;         /* dynamic Kn: the pressure of a node is p0 (1 + kn_beta
                             (rho - rho0)), its Kn = Kn(p0) p0 / p; 0: static Kn */
} orc_params;

typedef struct orc_sim {
  orc_params p;
  double *f;    /* post-stream populations at the current time level */
  double *fs;   /* post-collision scratch */
  double *eps;  /* porosity per node */
  double *ka;   /* apparent permeability per node at rho0 (may be +inf) */
  double *ki;   /* intrinsic permeability per node (dynamic Kn) */
  double *kn;   /* Knudsen number per node at rho0 (dynamic Kn) */
  int64_t steps;
} orc_sim;

/* ------------------------------------------------------------------ */
/* Eq. 6-7: Beskok-Karniadakis-Civan correction factor, b = -1.        */
/* ------------------------------------------------------------------ */
double orc_fc(double kn) {
  if (kn == 0.0) return 1.0; /* Kn^-0.4348 diverges; the limit is 1 */
  const double b = -1.0;
  double alpha = 1.358 / (1.0 + 0.170 * pow(kn, -0.4348)); /* Eq. 7 */
  return (1.0 + alpha * kn) * (1.0 + 4.0 * kn / (1.0 - b * kn)); /* Eq. 6 */
}

/* Eq. 3 with f_c of Eq. 6-7: k_a = k_i * f_c(Kn). */
double orc_apparent_permeability(double k_i, double kn) {
  return k_i * orc_fc(kn);
}

/* Eq. 4-5: Klinkenberg's first-order factor f_c = 1 + b_k / p = 1 + 4 c Kn,
 * with c = 1. */
double orc_fc_first_order(double kn) { return 1.0 + 4.0 * kn; }

/* f_c of the model selected in the parameters. */
static double orc_fc_model(double kn, int32_t model) {
  return model == 1 ? orc_fc_first_order(kn) : orc_fc(kn);
}

/* ------------------------------------------------------------------ */
/* Eq. 9-11: physical inputs of Kn (SI units in and out).               */
/* ------------------------------------------------------------------ */
/* Eq. 9: Kozeny-Carman intrinsic permeability [m^2] of packed spheres of
 * diameter d [m]: k_d = C eps^3 / (1 - eps)^2 with C = d^2 / 180. */
double orc_kozeny_carman(double eps, double d) {
  const double C = d * d / 180.0;
  return C * eps * eps * eps / ((1.0 - eps) * (1.0 - eps));
}

/* Eq. 10: mean free path [m] of a gas of viscosity mu [Pa s] at pressure p
 * [Pa], temperature T [K], molar mass M [kg/mol]. */
double orc_mean_free_path(double mu, double p, double T, double M) {
  const double R = 8.314462618; /* J / (mol K) */
  return mu / p * sqrt(3.14159265358979323846 * R * T / (2.0 * M));
}

/* Eq. 11 (Herd et al.): pore radius r [um] = 8.886e-2 sqrt(k [mD] / eps),
 * here from k_d in m^2 to r in m (1 mD = 9.869e-16 m^2). */
double orc_pore_radius(double k_d, double eps) {
  const double k_mD = k_d / 9.869e-16;
  return 8.886e-2 * sqrt(k_mD / eps) * 1e-6;
}

/* Lattice viscosities: nu_e = c_s^2 (tau - 1/2) with c_s^2 = 1/3 (dt = 1),
 * nu = nu_e / J (Eq. 1b). */
static double orc_nu(const orc_params *p) { return (p->tau - 0.5) / 3.0 / p->J; }

/* ------------------------------------------------------------------ */
/* Macroscopic state of one node: Eq. 16a, Eq. 17 (or its quadratic    */
/* form with the Forchheimer term) and the total force of Eq. 2 / 8.   */
/* ------------------------------------------------------------------ */
void orc_node_state(const double *f, double eps, double ka,
                    const orc_params *p, double *rho_out, double *u_out,
                    double *F_out) {
  double rho = 0.0, mx = 0.0, my = 0.0;
  for (int i = 0; i < 9; ++i) { /* Eq. 16a and the sum in Eq. 16b */
    rho += f[i];
    mx += f[i] * ORC_EX[i];
    my += f[i] * ORC_EY[i];
  }
  double ux, uy, Fx, Fy;
  if (eps == 0.0) {
    /* impermeable node: infinite drag, u = 0; Eq. 16b then fixes F */
    ux = 0.0;
    uy = 0.0;
    Fx = -2.0 * mx / rho;
    Fy = -2.0 * my / rho;
  } else {
    const double nu = orc_nu(p);
    const double inv_k = 1.0 / ka; /* 0 for an open pore (ka = +inf) */
    if (!p->forchheimer) {
      /* Eq. 17 */
      double den = rho + 0.5 * (eps * nu / ka) * rho;
      ux = (mx + 0.5 * rho * eps * p->Gx) / den;
      uy = (my + 0.5 * rho * eps * p->Gy) / den;
      /* Eq. 8 */
      Fx = -(eps * nu / ka) * ux + eps * p->Gx;
      Fy = -(eps * nu / ka) * uy + eps * p->Gy;
    } else {
      /* Eq. 16b with the full drag of Eq. 2 is quadratic in |u|:
       *   u (A + B|u|) = v,  v = m/rho + eps G / 2,
       *   A = 1 + eps nu / (2 k),  B = eps F_eps / (2 sqrt(k)),
       * whose positive root gives u = v / (c0 + sqrt(c0^2 + c1 |v|)) with
       * c0 = A / 2, c1 = B.  F_eps from Ergun's relation. */
      double Feps = 1.75 / sqrt(150.0 * eps * eps * eps);
      double vx = mx / rho + 0.5 * eps * p->Gx;
      double vy = my / rho + 0.5 * eps * p->Gy;
      double c0 = 0.5 * (1.0 + 0.5 * eps * nu * inv_k);
      double c1 = 0.5 * eps * Feps * sqrt(inv_k);
      double vmag = sqrt(vx * vx + vy * vy);
      double den = c0 + sqrt(c0 * c0 + c1 * vmag);
      ux = vx / den;
      uy = vy / den;
      /* Eq. 2 */
      double umag = sqrt(ux * ux + uy * uy);
      Fx = -(eps * nu * inv_k) * ux - (eps * Feps * sqrt(inv_k)) * umag * ux +
           eps * p->Gx;
      Fy = -(eps * nu * inv_k) * uy - (eps * Feps * sqrt(inv_k)) * umag * uy +
           eps * p->Gy;
    }
  }
  if (rho_out) *rho_out = rho;
  if (u_out) { u_out[0] = ux; u_out[1] = uy; }
  if (F_out) { F_out[0] = Fx; F_out[1] = Fy; }
}

/* Eq. 14: porosity-weighted equilibrium (c = 1).  For eps = 0 the velocity
 * is zero and only the rest term w_i rho remains. */
void orc_feq(double rho, const double *u, double eps, double *feq) {
  for (int i = 0; i < 9; ++i) {
    if (eps == 0.0) {
      feq[i] = ORC_W[i] * rho;
      continue;
    }
    double eu = ORC_EX[i] * u[0] + ORC_EY[i] * u[1];
    double uu = u[0] * u[0] + u[1] * u[1];
    feq[i] = ORC_W[i] * rho *
             (1.0 + 3.0 * eu + 9.0 / (2.0 * eps) * eu * eu - 3.0 / (2.0 * eps) * uu);
  }
}

/* Eq. 15: Guo's forcing term, last term divided by eps (see header). */
void orc_forcing(double rho, const double *u, const double *F, double eps,
                 double tau, double *Fi) {
  for (int i = 0; i < 9; ++i) {
    double eF = ORC_EX[i] * F[0] + ORC_EY[i] * F[1];
    double bracket;
    if (eps == 0.0) {
      bracket = 3.0 * eF; /* u = 0: the u-terms vanish */
    } else {
      double eu = ORC_EX[i] * u[0] + ORC_EY[i] * u[1];
      double uF = u[0] * F[0] + u[1] * F[1];
      bracket = 3.0 * eF + 9.0 / eps * eu * eF - 3.0 / eps * uF;
    }
    Fi[i] = ORC_W[i] * rho * (1.0 - 1.0 / (2.0 * tau)) * bracket;
  }
}

/* Eq. 12 (right-hand side, dt = 1): the post-collision populations of one
 * node from its post-stream populations f. */
void orc_collide_node(const double *f, double eps, double ka,
                      const orc_params *p, double *fpost) {
  double rho, u[2], F[2], feq[9], Fi[9];
  orc_node_state(f, eps, ka, p, &rho, u, F);
  orc_feq(rho, u, eps, feq);
  orc_forcing(rho, u, F, eps, p->tau, Fi);
  for (int i = 0; i < 9; ++i)
    fpost[i] = f[i] - (f[i] - feq[i]) / p->tau + Fi[i];
}

/* Non-equilibrium extrapolation for a pressure boundary node b with imposed
 * density rho_b from its interior neighbour n (both post-stream):
 *   f_b = f_eq(rho_b, u_n; eps_b) + (f_n - f_eq(rho_n, u_n; eps_n)). */
void orc_neep_node(const double *fn, double eps_n, double ka_n, double eps_b,
                   double rho_b, const orc_params *p, double *fb) {
  double rho_n, u_n[2], feq_n[9], feq_b[9];
  orc_node_state(fn, eps_n, ka_n, p, &rho_n, u_n, NULL);
  orc_feq(rho_n, u_n, eps_n, feq_n);
  orc_feq(rho_b, u_n, eps_b, feq_b);
  for (int i = 0; i < 9; ++i) fb[i] = feq_b[i] + (fn[i] - feq_n[i]);
}

/* index of the velocity opposite to e_i */
static int orc_opposite(int i) {
  for (int j = 0; j < 9; ++j)
    if (ORC_EX[j] == -ORC_EX[i] && ORC_EY[j] == -ORC_EY[i]) return j;
  return -1;
}

static int orc_is_wall_row(const orc_params *p, int y) {
  return p->bc_y == ORC_BC_WALLS && (y == 0 || y == p->ny - 1);
}

/* Apparent permeability of node j whose post-stream populations are f:
 * the stored k_a, or with a dynamic Kn, k_i f_c(Kn(p0) p0 / p) with the
 * node's pressure p / p0 = 1 + kn_beta (rho - rho0), rho = sum f (Eq. 16a). */
static double orc_node_ka(const orc_sim *s, int64_t j, const double *f) {
  const orc_params *p = &s->p;
  if (p->kn_beta == 0.0) return s->ka[j];
  double rho = 0.0;
  for (int i = 0; i < 9; ++i) rho += f[i];
  const double q = 1.0 + p->kn_beta * (rho - p->rho0);
  return s->ki[j] * orc_fc_model(s->kn[j] / q, p->kn_model);
}

static void orc_apply_pressure(orc_sim *s) {
  const orc_params *p = &s->p;
  const int nx = p->nx, ny = p->ny;
  if (p->bc_x != ORC_BC_PRESSURE) return;
  for (int y = 0; y < ny; ++y) {
    if (orc_is_wall_row(p, y)) continue;
    int64_t b0 = (int64_t)y * nx, n0 = b0 + 1;
    int64_t b1 = (int64_t)y * nx + nx - 1, n1 = b1 - 1;
    orc_neep_node(s->f + n0 * 9, s->eps[n0], orc_node_ka(s, n0, s->f + n0 * 9), s->eps[b0],
                  p->rho_in, p, s->f + b0 * 9);
    orc_neep_node(s->f + n1 * 9, s->eps[n1], orc_node_ka(s, n1, s->f + n1 * 9), s->eps[b1],
                  p->rho_out, p, s->f + b1 * 9);
  }
}

/* ------------------------------------------------------------------ */
/* Simulation object                                                    */
/* ------------------------------------------------------------------ */
orc_sim *orc_create(const orc_params *p) {
  if (p->nx < 1 || p->ny < 1) return NULL;
  if (p->bc_x == ORC_BC_PRESSURE && p->nx < 3) return NULL;
  if (p->bc_y == ORC_BC_WALLS && p->ny < 3) return NULL;
  orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
  if (!s) return NULL;
  s->p = *p;
  size_t n = (size_t)p->nx * (size_t)p->ny;
  s->f = (double *)calloc(n * 9, sizeof(double));
  s->fs = (double *)calloc(n * 9, sizeof(double));
  s->eps = (double *)calloc(n, sizeof(double));
  s->ka = (double *)calloc(n, sizeof(double));
  s->ki = (double *)calloc(n, sizeof(double));
  s->kn = (double *)calloc(n, sizeof(double));
  if (!s->f || !s->fs || !s->eps || !s->ka || !s->ki || !s->kn) {
    free(s->f); free(s->fs); free(s->eps); free(s->ka); free(s->ki); free(s->kn); free(s);
    return NULL;
  }
  return s;
}

void orc_destroy(orc_sim *s) {
  if (!s) return;
  free(s->f); free(s->fs); free(s->eps); free(s->ka); free(s->ki); free(s->kn); free(s);
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Medium (row-major [ny][nx]): porosity, intrinsic permeability, Kn.  The
 * populations restart from rest at density rho0 (f_i = w_i rho0), with the
 * pressure columns extrapolated as at every other time level. */
void orc_set_fields(orc_sim *s, const double *eps, const double *k_i,
                    const double *kn) {
  const orc_params *p = &s->p;
  int64_t n = (int64_t)p->nx * p->ny;
  for (int64_t j = 0; j < n; ++j) {
    s->eps[j] = eps[j];
    s->ka[j] = k_i[j] * orc_fc_model(kn[j], p->kn_model); /* Eq. 3 */
    s->ki[j] = k_i[j];
    s->kn[j] = kn[j];
    for (int i = 0; i < 9; ++i) s->f[j * 9 + i] = ORC_W[i] * p->rho0;
  }
  s->steps = 0;
  orc_apply_pressure(s);
}

/* One time step of Eq. 12: collide every fluid node, push each population
 * to x + e_i, bounce back at walls, wrap periodic edges, then extrapolate the
 * pressure columns. */
void orc_step(orc_sim *s, int64_t nsteps) {
  const orc_params *p = &s->p;
  const int nx = p->nx, ny = p->ny;
  for (int64_t t = 0; t < nsteps; ++t) {
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
      if (orc_is_wall_row(p, y)) continue;
      for (int x = 0; x < nx; ++x) {
        int64_t j = (int64_t)y * nx + x;
        orc_collide_node(s->f + j * 9, s->eps[j], orc_node_ka(s, j, s->f + j * 9), p,
                         s->fs + j * 9);
      }
    }
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
      if (orc_is_wall_row(p, y)) continue;
      for (int x = 0; x < nx; ++x) {
        int64_t j = (int64_t)y * nx + x;
        /* gather form of the push: f_i(x) <- f*_i(x - e_i) */
        for (int i = 0; i < 9; ++i) {
          int xs = x - ORC_EX[i], ys = y - ORC_EY[i];
          int opp = orc_opposite(i);
          if (p->bc_y == ORC_BC_WALLS && (ys == 0 || ys == ny - 1)) {
            /* the population sent towards the wall returns reversed */
            s->f[j * 9 + i] = s->fs[j * 9 + opp];
            continue;
          }
          if (ys < 0) ys += ny;
          if (ys >= ny) ys -= ny;
          if (xs < 0 || xs >= nx) {
            if (p->bc_x == ORC_BC_PRESSURE) {
              s->f[j * 9 + i] = NAN; /* unknown: replaced by the extrapolation */
              continue;
            }
            xs = (xs + nx) % nx;
          }
          s->f[j * 9 + i] = s->fs[((int64_t)ys * nx + xs) * 9 + i];
        }
      }
    }
    orc_apply_pressure(s);
    s->steps++;
  }
}

int64_t orc_steps(const orc_sim *s) { return s->steps; }

/* Post-stream populations in plane-major layout [9][ny][nx]. */
void orc_get_populations(const orc_sim *s, double *out) {
  int64_t n = (int64_t)s->p.nx * s->p.ny;
  for (int64_t j = 0; j < n; ++j)
    for (int i = 0; i < 9; ++i) out[(int64_t)i * n + j] = s->f[j * 9 + i];
}

/* Overwrite the post-stream populations ([9][ny][nx]).  The result is a
 * time level, so the pressure columns are extrapolated again. */
void orc_set_populations(orc_sim *s, const double *in) {
  int64_t n = (int64_t)s->p.nx * s->p.ny;
  for (int64_t j = 0; j < n; ++j)
    for (int i = 0; i < 9; ++i) s->f[j * 9 + i] = in[(int64_t)i * n + j];
  orc_apply_pressure(s);
}

/* rho and the physical velocity (Eq. 16a, 17) of every node; wall rows
 * report zeros. */
void orc_macroscopic(const orc_sim *s, double *rho, double *ux, double *uy) {
  const orc_params *p = &s->p;
  for (int y = 0; y < p->ny; ++y)
    for (int x = 0; x < p->nx; ++x) {
      int64_t j = (int64_t)y * p->nx + x;
      if (orc_is_wall_row(p, y)) {
        rho[j] = ux[j] = uy[j] = 0.0;
        continue;
      }
      double r, u[2];
      orc_node_state(s->f + j * 9, s->eps[j], orc_node_ka(s, j, s->f + j * 9), p, &r, u, NULL);
      rho[j] = r;
      ux[j] = u[0];
      uy[j] = u[1];
    }
}

/* Driving gradient for Darcy's law over the whole domain.  The lattice
 * density carries eps p = c_s^2 rho (Eq. 1b), so an imposed density drop
 * rho_in - rho_out is a pressure drop c_s^2 (rho_in - rho_out) / eps; with a
 * heterogeneous medium eps is taken as the mean porosity of the fluid nodes.
 * G_eff = G_x + dp / (rho0 (nx - 1)), cf. G = dp / (L rho) in Section IV.A. */
double orc_driving_force(const orc_sim *s) {
  const orc_params *p = &s->p;
  double g = p->Gx;
  if (p->bc_x == ORC_BC_PRESSURE) {
    double se = 0.0;
    int64_t count = 0;
    for (int y = 0; y < p->ny; ++y) {
      if (orc_is_wall_row(p, y)) continue;
      for (int x = 0; x < p->nx; ++x) {
        se += s->eps[(int64_t)y * p->nx + x];
        count++;
      }
    }
    double eps_mean = se / (double)count;
    double dp = (p->rho_in - p->rho_out) / 3.0 / eps_mean;
    g += dp / (p->rho0 * (double)(p->nx - 1));
  }
  return g;
}

/* Global permeability: Darcy's law over the whole domain,
 * k_g = nu <u_x> / G_eff with <u_x> the mean superficial velocity over all
 * fluid nodes.  Returns k_g; *u_mean receives <u_x>. */
double orc_permeability(const orc_sim *s, double *u_mean) {
  const orc_params *p = &s->p;
  double sum = 0.0;
  int64_t count = 0;
  for (int y = 0; y < p->ny; ++y) {
    if (orc_is_wall_row(p, y)) continue;
    for (int x = 0; x < p->nx; ++x) {
      int64_t j = (int64_t)y * p->nx + x;
      double u[2];
      orc_node_state(s->f + j * 9, s->eps[j], orc_node_ka(s, j, s->f + j * 9), p, NULL, u,
                     NULL);
      sum += u[0];
      count++;
    }
  }
  double um = sum / (double)count;
  if (u_mean) *u_mean = um;
  return orc_nu(p) * um / orc_driving_force(s);
}

/* Total mass sum rho over fluid nodes. */
double orc_mass(const orc_sim *s) {
  const orc_params *p = &s->p;
  double m = 0.0;
  for (int y = 0; y < p->ny; ++y) {
    if (orc_is_wall_row(p, y)) continue;
    for (int x = 0; x < p->nx; ++x) {
      int64_t j = (int64_t)y * p->nx + x;
      for (int i = 0; i < 9; ++i) m += s->f[j * 9 + i];
    }
  }
  return m;
}

/* Relative velocity residual || u - u_prev ||_2 / || u ||_2 over fluid
 * nodes, u_prev given as [ny][nx] arrays (wall rows ignored). */
double orc_residual(const orc_sim *s, const double *ux_prev,
                    const double *uy_prev) {
  const orc_params *p = &s->p;
  double num = 0.0, den = 0.0;
  for (int y = 0; y < p->ny; ++y) {
    if (orc_is_wall_row(p, y)) continue;
    for (int x = 0; x < p->nx; ++x) {
      int64_t j = (int64_t)y * p->nx + x;
      double u[2];
      orc_node_state(s->f + j * 9, s->eps[j], orc_node_ka(s, j, s->f + j * 9), p, NULL, u,
                     NULL);
      double dx = u[0] - ux_prev[j], dy = u[1] - uy_prev[j];
      num += dx * dx + dy * dy;
      den += u[0] * u[0] + u[1] * u[1];
    }
  }
  return sqrt(num) / sqrt(den);
}

/* Lattice tables, exported so tests can check them against Eq. 13. */
void orc_lattice(int *ex, int *ey, double *w) {
  for (int i = 0; i < 9; ++i) {
    ex[i] = ORC_EX[i];
    ey[i] = ORC_EY[i];
    w[i] = ORC_W[i];
  }
}

/* ------------------------------------------------------------------ */
/* Gradient of the global permeability by central differences: the      */
/* definition of the derivative, no adjoint.  For each listed node j,    */
/*   out[m] = (k_g(theta + h e_j) - k_g(theta - h e_j)) / (2 h),         */
/* k_g after nsteps steps from rest, theta_j = ln k_i(j) (which = 0) or   */
/* eps(j) (which = 1), m the position of j in `nodes`.  Each evaluation  */
/* is a separate lattice; they run in parallel (the loops inside         */
/* orc_step are then nested regions and run serially).  Returns 0, or   */
/* -1 when a node index is out of range or memory runs out.              */
/* ------------------------------------------------------------------ */
int orc_kg_fd(const orc_params *p, const double *eps, const double *k_i,
              const double *kn, int64_t nsteps, double h,
              const int64_t *nodes, int64_t count, int which, double *out) {
  const int64_t n = (int64_t)p->nx * p->ny;
  double *kg = (double *)calloc((size_t)(2 * count + 1), sizeof(double));
  if (!kg) return -1;
  int failed = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : failed)
  for (int64_t e = 0; e < 2 * count; ++e) {
    const int64_t j = nodes[e / 2];
    const double sign = (e % 2 == 0) ? 1.0 : -1.0;
    double *pe = (double *)malloc((size_t)n * sizeof(double));
    double *pk = (double *)malloc((size_t)n * sizeof(double));
    orc_sim *s = orc_create(p);
    if (!pe || !pk || !s || j < 0 || j >= n) {
      failed |= 1;
    } else {
      memcpy(pe, eps, (size_t)n * sizeof(double));
      memcpy(pk, k_i, (size_t)n * sizeof(double));
      if (which == 0)
        pk[j] = k_i[j] * exp(sign * h);
      else
        pe[j] = eps[j] + sign * h;
      orc_set_fields(s, pe, pk, kn);
      orc_step(s, nsteps);
      kg[e] = orc_permeability(s, NULL);
    }
    orc_destroy(s);
    free(pe);
    free(pk);
  }
  if (!failed)
    for (int64_t m = 0; m < count; ++m) out[m] = (kg[2 * m] - kg[2 * m + 1]) / (2.0 * h);
  free(kg);
  return failed ? -1 : 0;
}

/* ------------------------------------------------------------------ */
/* Normalised velocity magnitude u0 = |u| / max |u| over every node of  */
/* the fluid rows (Section IV.B, Fig. 6), counted in nbins equal ranges */
/* of [0, 1] (u0 = 1 falls in the last one; max |u| = 0 puts every node */
/* in the first).  *umax receives max |u|.                              */
/* ------------------------------------------------------------------ */
void orc_velocity_histogram(const orc_sim *s, int nbins, int64_t *counts, double *umax) {
  const orc_params *p = &s->p;
  const int64_t n = (int64_t)p->nx * p->ny;
  double *speed = (double *)malloc((size_t)n * sizeof(double));
  double mx = 0.0;
  for (int k = 0; k < nbins; ++k) counts[k] = 0;
  if (!speed) {
    *umax = NAN;
    return;
  }
  for (int y = 0; y < p->ny; ++y) {
    if (orc_is_wall_row(p, y)) continue;
    for (int x = 0; x < p->nx; ++x) {
      const int64_t j = (int64_t)y * p->nx + x;
      double u[2];
      orc_node_state(s->f + j * 9, s->eps[j], orc_node_ka(s, j, s->f + j * 9), p, NULL, u, NULL);
      speed[j] = sqrt(u[0] * u[0] + u[1] * u[1]);
      if (speed[j] > mx) mx = speed[j];
    }
  }
  for (int y = 0; y < p->ny; ++y) {
    if (orc_is_wall_row(p, y)) continue;
    for (int x = 0; x < p->nx; ++x) {
      const int64_t j = (int64_t)y * p->nx + x;
      int k = 0;
      if (mx > 0.0) {
        k = (int)floor(speed[j] / mx * nbins);
        if (k > nbins - 1) k = nbins - 1;
      }
      counts[k]++;
    }
  }
  free(speed);
  *umax = mx;
}
