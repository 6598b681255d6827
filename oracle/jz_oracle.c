/*
 * jz_oracle.c -- plain CPU FP64 oracle for the stage residual and the explicit
 * 5-stage Runge-Kutta update of the filtered compressible Navier-Stokes (LES)
 * equations on a structured curvilinear grid, after "On the Scalability of CFD
 * Tool for Supersonic Jet Flow Configurations" (arXiv 2003.09926), Section 3.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The GPU product path
 * never calls it, and it shares no code, header, table or constant generator
 * with the CUDA sources.
 *
 * Style: every stage of the method is a separate sweep over whole arrays, in
 * the order the method states it, in double precision, with no blocking,
 * fusion or reordering.  Compile with -ffp-contract=off.
 *
 * Readings of passages the paper leaves silent or garbled are labelled R1..R13
 * (the same labels are used in the project's design notes):
 *   R1  non-dimensionalisation: rho_inf = c_inf = T_inf = D = 1, p_inf = 1/gamma,
 *       gas constant 1/gamma, Cp = 1/(gamma-1), T = gamma p / rho, c^2 = T,
 *       jet U_j = M, mu_inf = U_j D / Re.
 *   R2  Eq. 2: e is total energy per unit VOLUME (the formula's dimensions).
 *   R3  Sutherland (Eq. sutherland): mu = mu_inf T^{3/2} (1+S1)/(T+S1), T_inf = 1.
 *   R4  tanh clustering of y and z about |y| = r_c.
 *   R5  seeded sinusoidal offset mapping of the coordinates.
 *   R6  metric terms in the conservative (Thomas-Lombard) form.
 *   R7  jet initial state: top-hat profile plus seeded velocity noise.
 *   R8  boundary nodes set at each stage start; Riemann far field from the
 *       nearest interior node; face priority x- > x+ > z+ > z- > y+ > y-;
 *       ghost layers copy (zeroth order) or wrap (periodic).
 *   R9  Turkel-Vatsa constants k2 = 1/4, k4 = 1/256, sigma = 1/2, sensor
 *       maximum taken over the two nodes of a face.
 *   R10 SGS model: Smagorinsky, Delta = J^{-1/3}, C_s = 0.18, Pr_t = 0.9;
 *       optionally Vreman's model with c = 2.5 C_s^2 and the same Delta.
 *   R11 Jameson 5-stage coefficients alpha = (1/4, 1/6, 3/8, 1/2, 1).
 *   R12 time step from a CFL number and the convective + viscous spectral radii.
 *   R14 cylindrical grid (Section 3): xi axial, eta radial from the centreline
 *       r = 0, zeta azimuthal with nk points whose first and last coincide
 *       (period P = nk - 1, P even).  Centreline nodes: the conserved
 *       variables of the adjacent radial node line (eta = 1) averaged over the
 *       P distinct azimuthal nodes, summed in azimuthal order (zeroth-order
 *       extrapolation, then the average); ghost nodes behind the centreline
 *       are the nodes across it, (xi, -eta, zeta + P/2); the last azimuthal
 *       plane is a copy of the first.
 *   R15 the conservative metric form gives zero volume (1/J = 0) on the
 *       centreline; J there is taken from the node at eta = 1.  The
 *       centreline's eta-flux enters its neighbours through S^eta, which
 *       vanishes there, so J only affects the time-step bound and the
 *       diagnostics' volume weights.  A far-field node on the centreline
 *       takes its outward normal from the node at eta = 1.  Where a
 *       directional spectral radius
 *       is zero its anisotropic scaling is zero (the limit for sigma < 1).
 *
 * Array layout (private to the oracle): every field is a dense array over the
 * padded box (ni+4) x (nj+4) x (nk+4) (two ghost layers on every face),
 * i fastest.  Multi-component fields are component-major.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NG 2
#define PI 3.14159265358979323846

enum { BC_PERIODIC = 0, BC_INFLOW = 1, BC_FARFIELD = 2, BC_AXIS = 4 };
enum { GEOM_BOX = 0, GEOM_CYLINDER = 1 };
enum { IC_JET = 0, IC_QUIESCENT = 1 };

typedef struct {
  int ni, nj, nk;
  int bc[6];            /* faces x-, x+, y-, y+, z-, z+ */
  double lo[3], hi[3];  /* domain extent per direction */
  double cluster_r;     /* R4: clustering radius r_c */
  double stretch_c;     /* R4: clustering strength c (0 = uniform) */
  double stretch_w;     /* R4: clustering width w */
  double map_amp;       /* R5: offset amplitude in units of the local spacing */
  uint64_t map_seed;    /* R5: seed of the mapping's integers and phases */
  int geom;             /* GEOM_BOX or GEOM_CYLINDER (R14) */
} orc_grid;

typedef struct {
  double mach, re, gamma, pr, prt, cs, k2, k4, sigma, s1, r0, theta, noise;
  int ic;
  int sgs; /* R10: 0 Smagorinsky, 1 Vreman */
} orc_flow;

/* ------------------------------------------------------------------------ */
/* indexing                                                                   */
/* ------------------------------------------------------------------------ */

static int ndim(const orc_grid* g, int d) { return d == 0 ? g->ni : (d == 1 ? g->nj : g->nk); }
static int is_periodic(const orc_grid* g, int d) { return g->bc[2 * d] == BC_PERIODIC; }
static ptrdiff_t pext(const orc_grid* g, int d) { return ndim(g, d) + 2 * NG; }

size_t orc_npad(const orc_grid* g) {
  return (size_t)pext(g, 0) * (size_t)pext(g, 1) * (size_t)pext(g, 2);
}

static size_t at(const orc_grid* g, int i, int j, int k) {
  return (size_t)(i + NG) + (size_t)pext(g, 0) * ((size_t)(j + NG) + (size_t)pext(g, 1) * (size_t)(k + NG));
}

static ptrdiff_t stride(const orc_grid* g, int d) {
  return d == 0 ? 1 : (d == 1 ? pext(g, 0) : pext(g, 0) * pext(g, 1));
}

static int is_cyl(const orc_grid* g) { return g->geom == GEOM_CYLINDER; }

/* number of distinct nodes of a periodic direction: n, or n - 1 for the
 * azimuthal direction of a cylindrical grid (first and last coincide, R14) */
static int period(const orc_grid* g, int d) { return (is_cyl(g) && d == 2) ? ndim(g, d) - 1 : ndim(g, d); }

/* lowest / highest node that receives the Runge-Kutta update (R8, R14) */
static int interior_lo(const orc_grid* g, int d) { return is_periodic(g, d) ? 0 : 1; }
static int interior_hi(const orc_grid* g, int d) { return is_periodic(g, d) ? period(g, d) - 1 : ndim(g, d) - 2; }

/* the grid node whose value a ghost index holds: wrap or clamp (R8) */
static int map_index(const orc_grid* g, int d, int idx) {
  int n = ndim(g, d);
  if (is_periodic(g, d)) {
    int P = period(g, d);
    return ((idx % P) + P) % P;
  }
  if (idx < 0) return 0;
  if (idx > n - 1) return n - 1;
  return idx;
}

/* the grid node a padded index (i, j, k) holds: behind the centreline of a
 * cylindrical grid the node across it (R14), else direction by direction */
static void map_node(const orc_grid* g, int* i, int* j, int* k) {
  if (is_cyl(g) && *j < 0) {
    *j = -*j;
    *k += period(g, 2) / 2;
  }
  *i = map_index(g, 0, *i);
  *j = map_index(g, 1, *j);
  *k = map_index(g, 2, *k);
}

/* ------------------------------------------------------------------------ */
/* counter-based generator: SplitMix64 (Steele, Lea & Flood 2014)             */
/* ------------------------------------------------------------------------ */

/* First output of a SplitMix64 generator whose state is x. */
uint64_t orc_splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* uniform double in [0,1) from the top 53 bits */
static double unit53(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

/* ------------------------------------------------------------------------ */
/* grid: coordinates (R4, R5) and metric terms (R6)                           */
/* ------------------------------------------------------------------------ */

/* R5: integer wave numbers m in {1,2,3} and phases in [0, 2 pi) */
void orc_map_params(const orc_grid* g, int* m /* 9 */, double* th /* 9 */) {
  for (int d = 0; d < 3; ++d)
    for (int e = 0; e < 3; ++e) {
      uint64_t c = (uint64_t)(3 * d + e);
      m[3 * d + e] = 1 + (int)(orc_splitmix64(g->map_seed ^ (2 * c)) % 3ULL);
      th[3 * d + e] = 2.0 * PI * unit53(orc_splitmix64(g->map_seed ^ (2 * c + 1)));
    }
}

/* R4: odd, monotone stretching function with clustering about s = +-r_c/H */
static double stretch_G(const orc_grid* g, double H, double s) {
  return s - (g->stretch_c / H) * (tanh((H * s - g->cluster_r) / g->stretch_w) +
                                   tanh((H * s + g->cluster_r) / g->stretch_w));
}

/* unmapped coordinate of direction d at (possibly ghost) index idx; on a
 * cylindrical grid direction 1 gives the radius r in [0, hi[1]] (the same
 * odd clustering function on s = j / (nj - 1), so r(-j) = -r(j)) and
 * direction 2 the azimuth 2 pi (k mod P) / P */
double orc_base_coord(const orc_grid* g, int d, double idx) {
  int n = ndim(g, d);
  double lo = g->lo[d], hi = g->hi[d];
  if (is_cyl(g) && d == 1) {
    double s = idx / (n - 1);
    if (g->stretch_c == 0.0) return hi * s;
    return hi * stretch_G(g, hi, s) / stretch_G(g, hi, 1.0);
  }
  if (is_cyl(g) && d == 2) {
    int P = period(g, 2), kk = (int)idx;
    return 2.0 * PI * (double)(((kk % P) + P) % P) / P;
  }
  if (is_periodic(g, d)) return lo + (hi - lo) * idx / n;
  if (d == 0 || g->stretch_c == 0.0) return lo + (hi - lo) * idx / (n - 1);
  double H = 0.5 * (hi - lo), C = 0.5 * (hi + lo);
  double s = -1.0 + 2.0 * idx / (n - 1);
  return C + H * stretch_G(g, H, s) / stretch_G(g, H, 1.0);
}

/* Coordinates x_d at every padded node (ghost indices are the analytic map at
 * the unwrapped index).  X is 3 x npad. */
void orc_coords(const orc_grid* g, double* X) {
  size_t np = orc_npad(g);
  int m[9];
  double th[9];
  orc_map_params(g, m, th);
#pragma omp parallel for schedule(static)
  for (int k = -NG; k < g->nk + NG; ++k)
    for (int j = -NG; j < g->nj + NG; ++j)
      for (int i = -NG; i < g->ni + NG; ++i) {
        int idx[3] = {i, j, k};
        if (is_cyl(g)) { /* R14: x axial, (y, z) = r (cos theta, sin theta) */
          double r = orc_base_coord(g, 1, j), th = orc_base_coord(g, 2, k);
          X[at(g, i, j, k)] = orc_base_coord(g, 0, i);
          X[np + at(g, i, j, k)] = r * cos(th);
          X[2 * np + at(g, i, j, k)] = r * sin(th);
          continue;
        }
        for (int d = 0; d < 3; ++d) {
          double base = orc_base_coord(g, d, idx[d]);
          double x = base;
          if (g->map_amp != 0.0) {
            double h = 0.5 * (orc_base_coord(g, d, idx[d] + 1.0) - orc_base_coord(g, d, idx[d] - 1.0));
            double prod = 1.0;
            for (int e = 0; e < 3; ++e) {
              int P = is_periodic(g, e) ? ndim(g, e) : ndim(g, e) - 1;
              prod *= sin(2.0 * PI * m[3 * d + e] * idx[e] / P + th[3 * d + e]);
            }
            x = base + g->map_amp * h * prod;
          }
          X[(size_t)d * np + at(g, i, j, k)] = x;
        }
      }
}

/* central difference (Delta xi = 1) of f along stride s at node n */
static double dc(const double* f, size_t n, ptrdiff_t s) { return 0.5 * (f[n + s] - f[n - s]); }

/* Fill the ghost entries of a multi-component node field by the node map. */
static void fill_ghosts(const orc_grid* g, double* F, int ncomp) {
  size_t np = orc_npad(g);
  for (int k = -NG; k < g->nk + NG; ++k)
    for (int j = -NG; j < g->nj + NG; ++j)
      for (int i = -NG; i < g->ni + NG; ++i) {
        int mi = i, mj = j, mk = k;
        map_node(g, &mi, &mj, &mk);
        if (mi == i && mj == j && mk == k) continue;
        for (int c = 0; c < ncomp; ++c)
          F[(size_t)c * np + at(g, i, j, k)] = F[(size_t)c * np + at(g, mi, mj, mk)];
      }
}

/* R6: conservative (Thomas-Lombard) metric terms.
 *   S[3*k+m] = (d xi_k / d x_m) / J, i.e. with (a,b,c) the cyclic order of
 *   the computational directions starting at k, and (m,p,q) the cyclic order
 *   of the Cartesian coordinates starting at m:
 *       S^k_m = d_c( d_b(x_p) x_q ) - d_b( d_c(x_p) x_q ),
 *   which gives sum_k d_k S^k_m = 0 exactly because central differences
 *   commute.  1/J = det(d x_m / d xi_k) from central differences.
 * Computed at every grid node 0..N-1, then ghost entries by the node map. */
void orc_metrics(const orc_grid* g, const double* X, double* S /* 9 x npad */, double* J) {
  size_t np = orc_npad(g);
#pragma omp parallel for schedule(static)
  for (int k = 0; k < g->nk; ++k)
    for (int j = 0; j < g->nj; ++j)
      for (int i = 0; i < g->ni; ++i) {
        size_t n = at(g, i, j, k);
        for (int kd = 0; kd < 3; ++kd) {
          ptrdiff_t sb = stride(g, (kd + 1) % 3), sc = stride(g, (kd + 2) % 3);
          for (int md = 0; md < 3; ++md) {
            const double* xp = X + (size_t)((md + 1) % 3) * np;
            const double* xq = X + (size_t)((md + 2) % 3) * np;
            double t1 = 0.5 * (dc(xp, n + sc, sb) * xq[n + sc] - dc(xp, n - sc, sb) * xq[n - sc]);
            double t2 = 0.5 * (dc(xp, n + sb, sc) * xq[n + sb] - dc(xp, n - sb, sc) * xq[n - sb]);
            S[(size_t)(3 * kd + md) * np + n] = t1 - t2;
          }
        }
        double A[3][3]; /* A[m][k] = d x_m / d xi_k */
        for (int md = 0; md < 3; ++md)
          for (int kd = 0; kd < 3; ++kd) A[md][kd] = dc(X + (size_t)md * np, n, stride(g, kd));
        double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
                     A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                     A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
        J[n] = 1.0 / det;
      }
  if (is_cyl(g)) /* R15: the centreline takes J of the adjacent radial node */
    for (int k = 0; k < g->nk; ++k)
      for (int i = 0; i < g->ni; ++i) J[at(g, i, 0, k)] = J[at(g, i, 1, k)];
  fill_ghosts(g, S, 9);
  fill_ghosts(g, J, 1);
}

/* ------------------------------------------------------------------------ */
/* gas model (Eq. 2, Eq. sutherland, equation of state; R1-R3)                */
/* ------------------------------------------------------------------------ */

double orc_mu_inf(const orc_flow* f) { return f->re > 0.0 ? f->mach / f->re : 0.0; }

/* R3: Sutherland law, temperature in units of T_inf */
double orc_sutherland(const orc_flow* f, double T) {
  return orc_mu_inf(f) * pow(T, 1.5) * (1.0 + f->s1) / (T + f->s1);
}

/* conserved -> primitive: rho, u, v, w, p, T */
static void primitives(const orc_flow* f, const double q[5], double w[6]) {
  double rho = q[0];
  double u = q[1] / rho, v = q[2] / rho, ww = q[3] / rho;
  double p = (f->gamma - 1.0) * (q[4] - 0.5 * rho * (u * u + v * v + ww * ww));
  w[0] = rho; w[1] = u; w[2] = v; w[3] = ww; w[4] = p;
  w[5] = f->gamma * p / rho;
}

static void conserved(const orc_flow* f, double rho, double u, double v, double w, double p, double q[5]) {
  q[0] = rho;
  q[1] = rho * u;
  q[2] = rho * v;
  q[3] = rho * w;
  q[4] = p / (f->gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w);
}

/* R7: top-hat jet profile (axial velocity) at radius r */
double orc_jet_profile(const orc_flow* f, double r) {
  return 0.5 * f->mach * (1.0 - tanh((r - f->r0) / (2.0 * f->theta)));
}

/* ------------------------------------------------------------------------ */
/* boundary conditions (R8)                                                   */
/* ------------------------------------------------------------------------ */

/* Riemann-invariant far field (1-D, normal to the face).  qi: interior state,
 * n: outward unit normal; exterior = freestream at rest (rho 1, u 0, p 1/gamma). */
void orc_riemann_farfield(const orc_flow* f, const double qi[5], const double n[3], double qb[5]) {
  double g = f->gamma;
  double wi[6];
  primitives(f, qi, wi);
  double rho_i = wi[0], p_i = wi[4];
  double ui[3] = {wi[1], wi[2], wi[3]};
  double c_i = sqrt(g * p_i / rho_i);
  double rho_e = 1.0, p_e = 1.0 / g, c_e = 1.0;
  double ue[3] = {0.0, 0.0, 0.0};
  double un_i = ui[0] * n[0] + ui[1] * n[1] + ui[2] * n[2];
  double un_e = ue[0] * n[0] + ue[1] * n[1] + ue[2] * n[2];
  if (un_i >= c_i) { /* supersonic outflow: everything from the interior */
    for (int v = 0; v < 5; ++v) qb[v] = qi[v];
    return;
  }
  if (un_i <= -c_i) { /* supersonic inflow: everything from outside */
    conserved(f, rho_e, ue[0], ue[1], ue[2], p_e, qb);
    return;
  }
  double Rp = un_i + 2.0 * c_i / (g - 1.0);
  double Rm = un_e - 2.0 * c_e / (g - 1.0);
  double un = 0.5 * (Rp + Rm);
  double c = 0.25 * (g - 1.0) * (Rp - Rm);
  double s, ut[3];
  if (un > 0.0) {
    s = p_i / pow(rho_i, g);
    for (int d = 0; d < 3; ++d) ut[d] = ui[d] - un_i * n[d];
  } else {
    s = p_e / pow(rho_e, g);
    for (int d = 0; d < 3; ++d) ut[d] = ue[d] - un_e * n[d];
  }
  double rho = pow(c * c / (g * s), 1.0 / (g - 1.0));
  double p = rho * c * c / g;
  conserved(f, rho, ut[0] + un * n[0], ut[1] + un * n[1], ut[2] + un * n[2], p, qb);
}

/* the face that sets a boundary node: later faces in the order
 * y-, y+, z-, z+, x+, x- overwrite earlier ones; -1 if none */
static int winning_face(const orc_grid* g, const int idx[3]) {
  static const int order[6] = {2, 3, 4, 5, 1, 0};
  int win = -1;
  for (int o = 0; o < 6; ++o) {
    int face = order[o], d = face / 2;
    if (g->bc[face] == BC_PERIODIC) continue;
    int target = (face % 2 == 0) ? 0 : ndim(g, d) - 1;
    if (idx[d] == target) win = face;
  }
  return win;
}

/* Set boundary nodes and ghost layers of Q (5 x npad). */
void orc_apply_bc(const orc_grid* g, const orc_flow* f, const double* X, const double* S, double* Q) {
  size_t np = orc_npad(g);
  /* boundary nodes: read only interior nodes, so the order of nodes is free */
#pragma omp parallel for schedule(static)
  for (int k = 0; k < g->nk; ++k)
    for (int j = 0; j < g->nj; ++j)
      for (int i = 0; i < g->ni; ++i) {
        int idx[3] = {i, j, k};
        int face = winning_face(g, idx);
        if (face < 0) continue;
        size_t n = at(g, i, j, k);
        double qb[5];
        if (g->bc[face] == BC_INFLOW) {
          double y = X[np + n], z = X[2 * np + n];
          conserved(f, 1.0, orc_jet_profile(f, sqrt(y * y + z * z)), 0.0, 0.0, 1.0 / f->gamma, qb);
        } else if (g->bc[face] == BC_AXIS) { /* R14: azimuthal mean of the eta = 1 line */
          int P = period(g, 2);
          for (int v = 0; v < 5; ++v) {
            double s = 0.0;
            for (int kk = 0; kk < P; ++kk) s += Q[(size_t)v * np + at(g, i, 1, kk)];
            qb[v] = s / P;
          }
        } else {
          int ci[3];
          for (int d = 0; d < 3; ++d) {
            ci[d] = idx[d];
            if (ci[d] < interior_lo(g, d)) ci[d] = interior_lo(g, d);
            if (ci[d] > interior_hi(g, d)) ci[d] = interior_hi(g, d);
          }
          size_t c = at(g, ci[0], ci[1], ci[2]);
          double qi[5], nrm[3];
          for (int v = 0; v < 5; ++v) qi[v] = Q[(size_t)v * np + c];
          int d = face / 2;
          double sgn = (face % 2 == 0) ? -1.0 : 1.0;
          /* R15: on the centreline the face metric vanishes; the normal is
           * that of the adjacent radial node */
          size_t nn = (is_cyl(g) && j == 0) ? at(g, i, 1, k) : n;
          double a = S[(size_t)(3 * d) * np + nn], b = S[(size_t)(3 * d + 1) * np + nn], cc = S[(size_t)(3 * d + 2) * np + nn];
          double len = sqrt(a * a + b * b + cc * cc);
          nrm[0] = sgn * a / len; nrm[1] = sgn * b / len; nrm[2] = sgn * cc / len;
          orc_riemann_farfield(f, qi, nrm, qb);
        }
        for (int v = 0; v < 5; ++v) Q[(size_t)v * np + n] = qb[v];
      }
  fill_ghosts(g, Q, 5);
}

/* ------------------------------------------------------------------------ */
/* initial state (R7)                                                         */
/* ------------------------------------------------------------------------ */

void orc_init(const orc_grid* g, const orc_flow* f, uint64_t seed, const double* X, const double* S, double* Q) {
  size_t np = orc_npad(g);
  memset(Q, 0, 5 * np * sizeof(double));
  for (int k = 0; k < g->nk; ++k)
    for (int j = 0; j < g->nj; ++j)
      for (int i = 0; i < g->ni; ++i) {
        size_t n = at(g, i, j, k);
        double u[3] = {0.0, 0.0, 0.0};
        if (f->ic == IC_JET) {
          double y = X[np + n], z = X[2 * np + n];
          u[0] = orc_jet_profile(f, sqrt(y * y + z * z));
          uint64_t lin = (uint64_t)i + (uint64_t)g->ni * ((uint64_t)j + (uint64_t)g->nj * (uint64_t)k);
          for (int m = 0; m < 3; ++m) {
            double xi = unit53(orc_splitmix64(seed ^ (3ULL * lin + (uint64_t)m)));
            u[m] += f->noise * f->mach * (2.0 * xi - 1.0);
          }
        }
        double q[5];
        conserved(f, 1.0, u[0], u[1], u[2], 1.0 / f->gamma, q);
        for (int v = 0; v < 5; ++v) Q[(size_t)v * np + n] = q[v];
      }
  orc_apply_bc(g, f, X, S, Q);
}

/* ------------------------------------------------------------------------ */
/* residual: inviscid flux, artificial dissipation, viscous flux + SGS        */
/* ------------------------------------------------------------------------ */

typedef struct {
  double* W;    /* 6 x npad primitives rho,u,v,w,p,T */
  double* Eh;   /* 15 x npad: contravariant inviscid flux E^k_v at [5k+v] */
  double* Fh;   /* 15 x npad: contravariant viscous flux F^k_v */
  double* lt;   /* 3 x npad: anisotropic spectral radius lambda~^k */
  double* nu;   /* 3 x npad: pressure sensor nu^k */
} work_t;

/* node range on which node quantities are formed: every node with a full
 * +-1 neighbourhood inside the padded box */
#define NODE_LOOP(g)                                   \
  for (int k = -1; k <= (g)->nk; ++k)                  \
    for (int j = -1; j <= (g)->nj; ++j)                \
      for (int i = -1; i <= (g)->ni; ++i)

static void sweep_primitives(const orc_grid* g, const orc_flow* f, const double* Q, double* W) {
  size_t np = orc_npad(g);
#pragma omp parallel for schedule(static)
  for (size_t n = 0; n < np; ++n) {
    double q[5], w[6];
    for (int v = 0; v < 5; ++v) q[v] = Q[(size_t)v * np + n];
    primitives(f, q, w);
    for (int c = 0; c < 6; ++c) W[(size_t)c * np + n] = w[c];
  }
}

/* Inviscid flux in computational direction k (Eq. con-prop, transformed):
 *   E^k = sum_m S^k_m E_m,  E_m = [rho u_m, rho u_i u_m + p delta_im, (e+p) u_m] */
static void sweep_inviscid(const orc_grid* g, const double* Q, const double* S, const double* W, double* Eh) {
  size_t np = orc_npad(g);
#pragma omp parallel for schedule(static)
  for (int k = -1; k <= g->nk; ++k)
    for (int j = -1; j <= g->nj; ++j)
      for (int i = -1; i <= g->ni; ++i) {
        size_t n = at(g, i, j, k);
        double rho = W[n], u[3] = {W[np + n], W[2 * np + n], W[3 * np + n]}, p = W[4 * np + n];
        double e = Q[4 * np + n];
        for (int kd = 0; kd < 3; ++kd) {
          double Sk[3] = {S[(size_t)(3 * kd) * np + n], S[(size_t)(3 * kd + 1) * np + n], S[(size_t)(3 * kd + 2) * np + n]};
          double E[5] = {0, 0, 0, 0, 0};
          for (int m = 0; m < 3; ++m) {
            double Em[5];
            Em[0] = rho * u[m];
            for (int ii = 0; ii < 3; ++ii) Em[1 + ii] = rho * u[ii] * u[m] + (ii == m ? p : 0.0);
            Em[4] = (e + p) * u[m];
            for (int v = 0; v < 5; ++v) E[v] += Sk[m] * Em[v];
          }
          for (int v = 0; v < 5; ++v) Eh[(size_t)(5 * kd + v) * np + n] = E[v];
        }
      }
}

/* Viscous flux with Smagorinsky or Vreman SGS viscosity (Eqs. q_mod,
 * sutherland, tau_mod; R10).  Cartesian gradients at the node:
 *   d phi / d x_m = J sum_k S^k_m d_k phi     (central d_k, Delta xi = 1)
 *   F_m = [0, tau_1m, tau_2m, tau_3m, u_i tau_im - q_m],  q_m = -kappa dT/dx_m
 *   F^k = sum_m S^k_m F_m */
static void sweep_viscous(const orc_grid* g, const orc_flow* f, const double* S, const double* J, const double* W,
                          double* Fh) {
  size_t np = orc_npad(g);
  double Cp = 1.0 / (f->gamma - 1.0);
#pragma omp parallel for schedule(static)
  for (int k = -1; k <= g->nk; ++k)
    for (int j = -1; j <= g->nj; ++j)
      for (int i = -1; i <= g->ni; ++i) {
        size_t n = at(g, i, j, k);
        /* computational derivatives of u, v, w, T (primitive slots 1, 2, 3, 5) */
        static const int slot[4] = {1, 2, 3, 5};
        double dxi[4][3];
        for (int c = 0; c < 4; ++c)
          for (int kd = 0; kd < 3; ++kd) dxi[c][kd] = dc(W + (size_t)slot[c] * np, n, stride(g, kd));
        /* Cartesian gradients grad[c][m] */
        double grad[4][3];
        for (int c = 0; c < 4; ++c)
          for (int m = 0; m < 3; ++m) {
            double s = 0.0;
            for (int kd = 0; kd < 3; ++kd) s += S[(size_t)(3 * kd + m) * np + n] * dxi[c][kd];
            grad[c][m] = J[n] * s;
          }
        double rho = W[n], T = W[5 * np + n];
        double u[3] = {W[np + n], W[2 * np + n], W[3 * np + n]};
        double delta = pow(J[n], -1.0 / 3.0);
        double mu_t;
        if (f->sgs == 1) {
          /* Vreman: alpha_ij = du_j/dx_i = grad[j][i], beta = Delta^2 alpha^T alpha,
           * B_beta = sum of the principal 2x2 minors of beta,
           * mu_t = rho c sqrt(B_beta / (alpha_ij alpha_ij)), c = 2.5 C_s^2 */
          double beta[3][3], aa = 0.0;
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
              double s = 0.0;
              for (int m = 0; m < 3; ++m) s += grad[a][m] * grad[b][m]; /* alpha_ma alpha_mb */
              beta[a][b] = delta * delta * s;
              aa += grad[a][b] * grad[a][b];
            }
          double Bb = beta[0][0] * beta[1][1] - beta[0][1] * beta[0][1] + beta[0][0] * beta[2][2] -
                      beta[0][2] * beta[0][2] + beta[1][1] * beta[2][2] - beta[1][2] * beta[1][2];
          mu_t = aa > 0.0 ? rho * 2.5 * f->cs * f->cs * sqrt(fmax(Bb, 0.0) / aa) : 0.0;
        } else {
          /* Smagorinsky */
          double Sm2 = 0.0;
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
              double sab = 0.5 * (grad[a][b] + grad[b][a]);
              Sm2 += sab * sab;
            }
          double Smag = sqrt(2.0 * Sm2);
          mu_t = rho * (f->cs * delta) * (f->cs * delta) * Smag;
        }
        double mu = orc_sutherland(f, T);
        double mu_e = mu + mu_t;
        double kappa = Cp * (mu / f->pr + mu_t / f->prt);
        double div = grad[0][0] + grad[1][1] + grad[2][2];
        double tau[3][3];
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b)
            tau[a][b] = mu_e * (grad[a][b] + grad[b][a] - (a == b ? 2.0 / 3.0 * div : 0.0));
        for (int kd = 0; kd < 3; ++kd) {
          double F[5] = {0, 0, 0, 0, 0};
          for (int m = 0; m < 3; ++m) {
            double Fm[5];
            Fm[0] = 0.0;
            for (int a = 0; a < 3; ++a) Fm[1 + a] = tau[a][m];
            double q_m = -kappa * grad[3][m];
            Fm[4] = u[0] * tau[0][m] + u[1] * tau[1][m] + u[2] * tau[2][m] - q_m;
            for (int v = 0; v < 5; ++v) F[v] += S[(size_t)(3 * kd + m) * np + n] * Fm[v];
          }
          for (int v = 0; v < 5; ++v) Fh[(size_t)(5 * kd + v) * np + n] = F[v];
        }
      }
}

/* Directional spectral radii |S^k . u| + c |S^k|, their anisotropic scaling
 * (Turkel & Vatsa), lambda~^k = lambda^k (1 + sum_{k' != k} (lambda^k'/lambda^k)^sigma),
 * and the pressure sensor nu^k = |p+ - 2p + p-| / (p+ + 2p + p-). */
static void sweep_dissipation_coeffs(const orc_grid* g, const orc_flow* f, const double* S, const double* W,
                                     double* lt, double* nu) {
  size_t np = orc_npad(g);
#pragma omp parallel for schedule(static)
  for (int k = -1; k <= g->nk; ++k)
    for (int j = -1; j <= g->nj; ++j)
      for (int i = -1; i <= g->ni; ++i) {
        size_t n = at(g, i, j, k);
        double u[3] = {W[np + n], W[2 * np + n], W[3 * np + n]};
        double c = sqrt(W[5 * np + n]);
        double lam[3];
        for (int kd = 0; kd < 3; ++kd) {
          double a = S[(size_t)(3 * kd) * np + n], b = S[(size_t)(3 * kd + 1) * np + n], cc = S[(size_t)(3 * kd + 2) * np + n];
          lam[kd] = fabs(a * u[0] + b * u[1] + cc * u[2]) + c * sqrt(a * a + b * b + cc * cc);
        }
        for (int kd = 0; kd < 3; ++kd) {
          double sum = 1.0;
          for (int o = 0; o < 3; ++o)
            if (o != kd && lam[kd] > 0.0) sum += pow(lam[o] / lam[kd], f->sigma);
          lt[(size_t)kd * np + n] = lam[kd] * sum; /* R15: 0 where lambda^k = 0 */
          ptrdiff_t s = stride(g, kd);
          const double* p = W + 4 * np;
          nu[(size_t)kd * np + n] = fabs(p[n + s] - 2.0 * p[n] + p[n - s]) / (p[n + s] + 2.0 * p[n] + p[n - s]);
        }
      }
}

/* Artificial dissipation flux on the face between node n and n + e_k:
 *   d = lambda~_face [eps2 (Q_{n+1} - Q_n) - eps4 (Q_{n+2} - 3 Q_{n+1} + 3 Q_n - Q_{n-1})]
 *   lambda~_face = (lambda~_n + lambda~_{n+1})/2, eps2 = k2 max(nu_n, nu_{n+1}),
 *   eps4 = max(0, k4 - eps2)   (R9) */
static double face_dissipation(const orc_flow* f, const double* Qv, const double* ltk, const double* nuk, size_t n,
                               ptrdiff_t s) {
  double lam = 0.5 * (ltk[n] + ltk[n + s]);
  double eps2 = f->k2 * (nuk[n] > nuk[n + s] ? nuk[n] : nuk[n + s]);
  double eps4 = f->k4 - eps2;
  if (eps4 < 0.0) eps4 = 0.0;
  return lam * (eps2 * (Qv[n + s] - Qv[n]) - eps4 * (Qv[n + 2 * s] - 3.0 * Qv[n + s] + 3.0 * Qv[n] - Qv[n - s]));
}

static int work_alloc(const orc_grid* g, work_t* w) {
  size_t np = orc_npad(g);
  w->W = (double*)calloc(6 * np, sizeof(double));
  w->Eh = (double*)calloc(15 * np, sizeof(double));
  w->Fh = (double*)calloc(15 * np, sizeof(double));
  w->lt = (double*)calloc(3 * np, sizeof(double));
  w->nu = (double*)calloc(3 * np, sizeof(double));
  return (w->W && w->Eh && w->Fh && w->lt && w->nu) ? 0 : -1;
}

static void work_free(work_t* w) {
  free(w->W); free(w->Eh); free(w->Fh); free(w->lt); free(w->nu);
}

/* R (5 x npad) at every interior node (zero elsewhere):
 *   R = sum_k [ d_k E^k - d_k F^k - (d^k_{n+1/2} - d^k_{n-1/2}) ],
 * so that dQ/dt = -J R  (Eq. vec-les in the transformed frame). */
int orc_residual(const orc_grid* g, const orc_flow* f, const double* S, const double* J, const double* Q, double* R) {
  size_t np = orc_npad(g);
  work_t w;
  if (work_alloc(g, &w)) { work_free(&w); return -1; }
  sweep_primitives(g, f, Q, w.W);
  sweep_inviscid(g, Q, S, w.W, w.Eh);
  sweep_viscous(g, f, S, J, w.W, w.Fh);
  sweep_dissipation_coeffs(g, f, S, w.W, w.lt, w.nu);
  memset(R, 0, 5 * np * sizeof(double));
#pragma omp parallel for schedule(static)
  for (int k = interior_lo(g, 2); k <= interior_hi(g, 2); ++k)
    for (int j = interior_lo(g, 1); j <= interior_hi(g, 1); ++j)
      for (int i = interior_lo(g, 0); i <= interior_hi(g, 0); ++i) {
        size_t n = at(g, i, j, k);
        for (int v = 0; v < 5; ++v) {
          double r = 0.0;
          for (int kd = 0; kd < 3; ++kd) {
            ptrdiff_t s = stride(g, kd);
            const double* E = w.Eh + (size_t)(5 * kd + v) * np;
            const double* F = w.Fh + (size_t)(5 * kd + v) * np;
            const double* Qv = Q + (size_t)v * np;
            double dplus = face_dissipation(f, Qv, w.lt + (size_t)kd * np, w.nu + (size_t)kd * np, n, s);
            double dminus = face_dissipation(f, Qv, w.lt + (size_t)kd * np, w.nu + (size_t)kd * np, n - s, s);
            r += 0.5 * (E[n + s] - E[n - s]) - 0.5 * (F[n + s] - F[n - s]) - (dplus - dminus);
          }
          R[(size_t)v * np + n] = r;
        }
      }
  work_free(&w);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* time step (R12) and Runge-Kutta update (R11)                               */
/* ------------------------------------------------------------------------ */

/* max over grid nodes of  sum_k J lambda^k + 2 nu_max J^2 sum_k |S^k|^2,
 * nu_max = max(4/3, gamma/Pr) mu(T) / rho */
double orc_max_rate(const orc_grid* g, const orc_flow* f, const double* S, const double* J, const double* Q) {
  size_t np = orc_npad(g);
  double vfac = (4.0 / 3.0 > f->gamma / f->pr) ? 4.0 / 3.0 : f->gamma / f->pr;
  double best = 0.0; /* a maximum: the same in any order */
#pragma omp parallel for schedule(static) reduction(max : best)
  for (int k = 0; k < g->nk; ++k)
    for (int j = 0; j < g->nj; ++j)
      for (int i = 0; i < g->ni; ++i) {
        size_t n = at(g, i, j, k);
        double q[5], w[6];
        for (int v = 0; v < 5; ++v) q[v] = Q[(size_t)v * np + n];
        primitives(f, q, w);
        double c = sqrt(w[5]);
        double nu_max = vfac * orc_sutherland(f, w[5]) / w[0];
        double conv = 0.0, s2 = 0.0;
        for (int kd = 0; kd < 3; ++kd) {
          double a = S[(size_t)(3 * kd) * np + n], b = S[(size_t)(3 * kd + 1) * np + n], cc = S[(size_t)(3 * kd + 2) * np + n];
          double sq = a * a + b * b + cc * cc;
          conv += J[n] * (fabs(a * w[1] + b * w[2] + cc * w[3]) + c * sqrt(sq));
          s2 += sq;
        }
        double rate = conv + 2.0 * nu_max * J[n] * J[n] * s2;
        if (rate > best) best = rate;
      }
  return best;
}

static const double RK_ALPHA[5] = {1.0 / 4.0, 1.0 / 6.0, 3.0 / 8.0, 1.0 / 2.0, 1.0};

double orc_rk_alpha(int l) { return RK_ALPHA[l]; }

/* One time step.  Q (5 x npad) enters with boundary conditions applied and
 * leaves as Q^{n+1} with boundary conditions applied.  dt = cfl / max_rate
 * when cfl > 0, else dt_fixed.  Returns dt, or -1 on allocation failure. */
double orc_rk_step(const orc_grid* g, const orc_flow* f, const double* X, const double* S, const double* J, double* Q,
                   double cfl, double dt_fixed) {
  size_t np = orc_npad(g);
  double dt = cfl > 0.0 ? cfl / orc_max_rate(g, f, S, J, Q) : dt_fixed;
  double* Q0 = (double*)malloc(5 * np * sizeof(double));
  double* R = (double*)malloc(5 * np * sizeof(double));
  if (!Q0 || !R) { free(Q0); free(R); return -1.0; }
  memcpy(Q0, Q, 5 * np * sizeof(double));
  for (int l = 0; l < 5; ++l) {
    /* Q holds Q^(l-1); boundary nodes are set at the start of every stage */
    orc_apply_bc(g, f, X, S, Q);
    if (orc_residual(g, f, S, J, Q, R)) { free(Q0); free(R); return -1.0; }
#pragma omp parallel for schedule(static)
    for (int k = interior_lo(g, 2); k <= interior_hi(g, 2); ++k)
      for (int j = interior_lo(g, 1); j <= interior_hi(g, 1); ++j)
        for (int i = interior_lo(g, 0); i <= interior_hi(g, 0); ++i) {
          size_t n = at(g, i, j, k);
          for (int v = 0; v < 5; ++v)
            Q[(size_t)v * np + n] = Q0[(size_t)v * np + n] - RK_ALPHA[l] * dt * J[n] * R[(size_t)v * np + n];
        }
  }
  orc_apply_bc(g, f, X, S, Q);
  free(Q0);
  free(R);
  return dt;
}

/* ------------------------------------------------------------------------ */
/* diagnostics                                                                */
/* ------------------------------------------------------------------------ */

/* out[0..4]  sum over grid nodes of Q_v / J (sequential order: i, then j, then k)
 * out[5..6]  min / max rho;  out[7..8] min / max p;  out[9] max |u|/c
 * out[10]    number of grid nodes with a non-finite conserved value */
void orc_diagnostics(const orc_grid* g, const orc_flow* f, const double* J, const double* Q, double* out) {
  size_t np = orc_npad(g);
  double sum[5] = {0, 0, 0, 0, 0};
  double rmin = INFINITY, rmax = -INFINITY, pmin = INFINITY, pmax = -INFINITY, mmax = 0.0, bad = 0.0;
  for (int k = 0; k < g->nk; ++k)
    for (int j = 0; j < g->nj; ++j)
      for (int i = 0; i < g->ni; ++i) {
        size_t n = at(g, i, j, k);
        double q[5], w[6];
        int finite = 1;
        for (int v = 0; v < 5; ++v) {
          q[v] = Q[(size_t)v * np + n];
          if (!isfinite(q[v])) finite = 0;
        }
        if (!finite) { bad += 1.0; continue; }
        for (int v = 0; v < 5; ++v) sum[v] += q[v] / J[n];
        primitives(f, q, w);
        if (w[0] < rmin) rmin = w[0];
        if (w[0] > rmax) rmax = w[0];
        if (w[4] < pmin) pmin = w[4];
        if (w[4] > pmax) pmax = w[4];
        double mach = sqrt(w[1] * w[1] + w[2] * w[2] + w[3] * w[3]) / sqrt(w[5]);
        if (mach > mmax) mmax = mach;
      }
  for (int v = 0; v < 5; ++v) out[v] = sum[v];
  out[5] = rmin; out[6] = rmax; out[7] = pmin; out[8] = pmax; out[9] = mmax; out[10] = bad;
}

int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}
