/*
 * g4oracle.c -- plain, slow FP64 CPU oracle for Geant4-style navigation and
 * the simple gamma transport of Seiskari, Kommeri and Niemi, "GPU in Physics
 * Computation: Case Geant4 Navigation" (arXiv:1209.5235).
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the CPU-baseline
 * leg of the benchmark load this file's shared library; the CUDA library
 * never links, includes or calls it, and it shares no code with it.
 *
 * What it computes (the plain definitions, no acceleration structures):
 *  - locate (Sec. 3.2, first navigation problem): descend from the world,
 *    entering the first daughter, in placement order, that contains the
 *    point under the direction-aware Inside rule;
 *  - compute_step (Sec. 3.2, second navigation problem): minimum over the
 *    current volume's DistanceToOut and every daughter's DistanceToIn, with
 *    fixed tie rules; brute-force isotropic safety;
 *  - transport: Algorithm 1 (Sec. 3.1) -- Y = -log W, walk boundary to
 *    boundary accumulating S_j = S_{j-1} + (t_j - t_{j-1}) mu_j, interact at
 *    T = t_{j-1} + (Y - S_{j-1}) / mu_j (Eqs. 6-7) -- extended with Compton
 *    scattering (Kahn's rejection method for the Klein-Nishina law),
 *    photoabsorption, an energy cutoff and per-volume energy deposits;
 *  - free_path: Algorithm 1 exactly, returning T for a given Y.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key =
 * 64-bit seed, counter = (block, track id lo, track id hi, stream).  Two
 * uniforms in (0, 1] per block (from x1:x0 and x3:x2); every draw site takes
 * whole blocks.  Written here from the published definition.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -fopenmp -shared -fPIC.
 * Every floating-point operation is an IEEE double operation evaluated in
 * source order; the only transcendental functions are log (Y = -log W and the
 * Gaussian spot), exp (log-uniform energies) and sqrt.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define O_DMAX 32
#define O_MAXG 4096
#define O_INF INFINITY

enum { O_BOX = 0, O_TUBE = 1, O_ORB = 2, O_CONE = 3 };
enum { EV_NONE = 0, EV_PHOTO = 1, EV_COMPTON = 2, EV_CUTOFF = 3, EV_ESCAPE = 4, EV_PUSH = 5, EV_STEPLIMIT = 6 };
enum { LIM_PHYS = -2, LIM_MOTHER = -1, LIM_PUSH = -3, LIM_STEPLIMIT = -4 };
enum {
  C_TRACKS = 0, C_STEPS, C_GEOM, C_PHYS, C_PHOTO, C_COMPTON, C_ESCAPED, C_CUTOFF, C_PUSH, C_STEPLIMIT,
  C_DIST_IN, C_INSIDE, O_NCOUNT = 16
};

/* Solids: box, orb, tube segment and (full) cone, each in its own frame.
 * Tolerance: kTol = 1e-9 mm x scale; surface band = +-kHalf. */
static double kTol = 1e-9, kHalf = 0.5e-9;

typedef struct {
  int kind;
  double a, b, c;            /* box: hx hy hz | tube: rmin rmax hz | orb: r */
  double sphi, dphi;         /* tube */
  int seg, wide;             /* tube: phi segment? segment wider than pi? */
  double cs, ss, ce, se;     /* tube: cos/sin of start and end angle */
  /* cone: radii R(z) = k z + c of the outer (o) and inner (i) surfaces, c = hz above,
   * cos of their half-opening angles (ca = 1 / sqrt(1 + k^2)), inner surface present */
  double ko, co, ki, ci, cao, cai;
  int has_in;
} OSolid;

typedef struct {
  int mother, solid, mat;
  double t[3], c, s;         /* local -> mother: p_m = R(theta) p_l + t */
  int first, ndau;           /* daughters: dau[first .. first+ndau) */
} OVol;

typedef struct {
  double rho;
  int n;
  double *E, *muC, *muP;
} OMat;

/* Uniform grid over a mother's bounding box (its own frame): cell (i, j, k) lists, in placement
 * order, the daughters whose bounding box grown by O_GRID_PAD overlaps it (see "uniform-grid
 * acceleration" below). */
typedef struct {
  int n[3];
  double lo[3], w[3];
  int *off;                  /* n0 n1 n2 + 1 offsets into lst */
  int *lst;
} OGrid;

typedef struct {
  OSolid *sol; int nsol, capsol;
  OVol *vol; int nvol, capvol;
  OMat *mat; int nmat, capmat;
  int *dau;                  /* daughter ids grouped by mother, in placement order */
  int finalized;
  OGrid **grid;              /* per volume: NULL or its daughters' grid (timing mode) */
  int use_grid;
} OGeom;

static OGeom *G[O_MAXG];
static int NG = 0;

void o_set_scale(double scale) { kTol = 1e-9 * scale; kHalf = 0.5 * kTol; }
double o_tolerance(void) { return kTol; }

/* ------------------------------------------------------------------ geometry */

int o_new_geom(void) {
  if (NG >= O_MAXG) return -1;
  OGeom *g = (OGeom *)calloc(1, sizeof(OGeom));
  G[NG] = g;
  return NG++;
}

void o_free_all(void) {
  for (int i = 0; i < NG; ++i) {
    OGeom *g = G[i];
    if (!g) continue;
    for (int m = 0; m < g->nmat; ++m) { free(g->mat[m].E); free(g->mat[m].muC); free(g->mat[m].muP); }
    if (g->grid) {
      for (int v = 0; v < g->nvol; ++v)
        if (g->grid[v]) { free(g->grid[v]->off); free(g->grid[v]->lst); free(g->grid[v]); }
      free(g->grid);
    }
    free(g->mat); free(g->sol); free(g->vol); free(g->dau); free(g);
    G[i] = NULL;
  }
  NG = 0;
}

#define GROW(ptr, n, cap, T) do { if ((n) >= (cap)) { (cap) = (cap) ? 2 * (cap) : 64; \
    (ptr) = (T *)realloc((ptr), (size_t)(cap) * sizeof(T)); } } while (0)

int o_add_material(int gi, double rho, int n, const double *E, const double *muC, const double *muP) {
  OGeom *g = G[gi];
  if (n < 2) return -1;
  for (int k = 1; k < n; ++k) if (!(E[k] > E[k - 1])) return -1;
  GROW(g->mat, g->nmat, g->capmat, OMat);
  OMat *m = &g->mat[g->nmat];
  m->rho = rho; m->n = n;
  m->E = (double *)malloc(n * sizeof(double));
  m->muC = (double *)malloc(n * sizeof(double));
  m->muP = (double *)malloc(n * sizeof(double));
  memcpy(m->E, E, n * sizeof(double)); memcpy(m->muC, muC, n * sizeof(double)); memcpy(m->muP, muP, n * sizeof(double));
  return g->nmat++;
}

/* params: box (hx, hy, hz); tube (rmin, rmax, hz, sphi, dphi); orb (r). */
int o_add_solid(int gi, int kind, const double *p) {
  OGeom *g = G[gi];
  OSolid s;
  memset(&s, 0, sizeof(s));
  s.kind = kind;
  if (kind == O_BOX) {
    s.a = p[0]; s.b = p[1]; s.c = p[2];
    if (!(s.a > kTol && s.b > kTol && s.c > kTol)) return -1;
  } else if (kind == O_ORB) {
    s.a = p[0];
    if (!(s.a > kTol)) return -1;
  } else if (kind == O_TUBE) {
    s.a = p[0]; s.b = p[1]; s.c = p[2]; s.sphi = p[3]; s.dphi = p[4];
    if (!(s.a >= 0.0 && (s.a == 0.0 || s.a > kTol) && s.b > s.a + kTol && s.c > kTol)) return -1;
    if (!(s.dphi > 0.0 && s.dphi <= 2.0 * M_PI + 1e-12)) return -1;
    s.seg = s.dphi < 2.0 * M_PI - 1e-12;
    s.wide = s.seg && s.dphi > M_PI;
    s.cs = cos(s.sphi); s.ss = sin(s.sphi);
    s.ce = cos(s.sphi + s.dphi); s.se = sin(s.sphi + s.dphi);
  } else if (kind == O_CONE) {
    /* p = rmin1, rmax1 (at z = -hz), rmin2, rmax2 (at z = +hz), hz; full in phi */
    const double rmin1 = p[0], rmax1 = p[1], rmin2 = p[2], rmax2 = p[3], hz = p[4];
    if (!(hz > kTol && rmax1 > rmin1 + kTol && rmax2 > rmin2 + kTol)) return -1;
    if (!((rmin1 == 0.0 && rmin2 == 0.0) || (rmin1 > kTol && rmin2 > kTol))) return -1;
    s.c = hz;
    s.ko = (rmax2 - rmax1) / (2.0 * hz);
    s.co = 0.5 * (rmax1 + rmax2);
    s.ki = (rmin2 - rmin1) / (2.0 * hz);
    s.ci = 0.5 * (rmin1 + rmin2);
    s.cao = 1.0 / sqrt(1.0 + s.ko * s.ko);
    s.cai = 1.0 / sqrt(1.0 + s.ki * s.ki);
    s.has_in = rmin1 > 0.0;
  } else {
    return -1;
  }
  GROW(g->sol, g->nsol, g->capsol, OSolid);
  g->sol[g->nsol] = s;
  return g->nsol++;
}

int o_add_volume(int gi, int mother, int solid, int mat, const double *t, double c, double s) {
  OGeom *g = G[gi];
  if (solid < 0 || solid >= g->nsol || mat < 0 || mat >= g->nmat) return -1;
  if (g->nvol == 0 ? mother != -1 : (mother < 0 || mother >= g->nvol)) return -1;
  GROW(g->vol, g->nvol, g->capvol, OVol);
  OVol *v = &g->vol[g->nvol];
  v->mother = mother; v->solid = solid; v->mat = mat;
  v->t[0] = t[0]; v->t[1] = t[1]; v->t[2] = t[2]; v->c = c; v->s = s;
  v->first = 0; v->ndau = 0;
  return g->nvol++;
}

/* Group daughters by mother (stable: placement order); reject trees deeper than O_DMAX. */
int o_finalize(int gi) {
  OGeom *g = G[gi];
  int n = g->nvol;
  if (n == 0) return -1;
  for (int i = 0; i < n; ++i) g->vol[i].ndau = 0;
  for (int i = 1; i < n; ++i) g->vol[g->vol[i].mother].ndau++;
  int acc = 0;
  for (int i = 0; i < n; ++i) { g->vol[i].first = acc; acc += g->vol[i].ndau; g->vol[i].ndau = 0; }
  free(g->dau);
  g->dau = (int *)malloc((size_t)(acc > 0 ? acc : 1) * sizeof(int));
  for (int i = 1; i < n; ++i) {
    OVol *m = &g->vol[g->vol[i].mother];
    g->dau[m->first + m->ndau++] = i;
  }
  for (int i = 0; i < n; ++i) {
    int d = 1, j = i;
    while (g->vol[j].mother >= 0) { j = g->vol[j].mother; ++d; }
    if (d > O_DMAX) return -2;
  }
  g->finalized = 1;
  return 0;
}

int o_n_volumes(int gi) { return G[gi]->nvol; }

/* mother frame -> local frame of volume v: p_l = R^T (p_m - t), v_l = R^T v_m. */
static void to_local(const OVol *v, const double *pm, const double *vm, double *pl, double *vl) {
  double dx = pm[0] - v->t[0], dy = pm[1] - v->t[1], dz = pm[2] - v->t[2];
  pl[0] = v->c * dx + v->s * dy;
  pl[1] = -v->s * dx + v->c * dy;
  pl[2] = dz;
  vl[0] = v->c * vm[0] + v->s * vm[1];
  vl[1] = -v->s * vm[0] + v->c * vm[1];
  vl[2] = vm[2];
}

/* ------------------------------------------------------------------ solids */
/* All solid routines work in the solid's local frame.  Inside is direction
 * aware: a point within +-kHalf of the surface belongs to the solid iff the
 * direction points strictly inward through every surface within the band. */

static int box_inside(const OSolid *s, const double *p, const double *v) {
  const double h[3] = {s->a, s->b, s->c};
  double m = -O_INF;
  for (int i = 0; i < 3; ++i) { double d = fabs(p[i]) - h[i]; if (d > m) m = d; }
  if (m > kHalf) return 0;
  if (m < -kHalf) return 1;
  for (int i = 0; i < 3; ++i)
    if (fabs(p[i]) - h[i] >= -kHalf && p[i] * v[i] >= 0.0) return 0;
  return 1;
}

/* Slab method.  A point on or outside a face and not moving towards the slab
 * centre never enters; a chord not longer than kHalf is a miss. */
static double box_dist_in(const OSolid *s, const double *p, const double *v) {
  const double h[3] = {s->a, s->b, s->c};
  for (int i = 0; i < 3; ++i)
    if (fabs(p[i]) - h[i] >= -kHalf && p[i] * v[i] >= 0.0) return O_INF;
  double tin = -O_INF, tout = O_INF;
  for (int i = 0; i < 3; ++i) {
    if (v[i] == 0.0) continue;
    double t1 = (-h[i] - p[i]) / v[i];
    double t2 = (h[i] - p[i]) / v[i];
    double lo = t1 < t2 ? t1 : t2, hi = t1 < t2 ? t2 : t1;
    if (lo > tin) tin = lo;
    if (hi < tout) tout = hi;
  }
  if (!(tout > tin + kHalf)) return O_INF;
  return tin > 0.0 ? tin : 0.0;
}

static double box_dist_out(const OSolid *s, const double *p, const double *v) {
  const double h[3] = {s->a, s->b, s->c};
  double t = O_INF;
  for (int i = 0; i < 3; ++i) {
    double ti;
    if (v[i] > 0.0) ti = (h[i] - p[i]) / v[i];
    else if (v[i] < 0.0) ti = (-h[i] - p[i]) / v[i];
    else continue;
    if (ti < t) t = ti;
  }
  return t > 0.0 ? t : 0.0;
}

static double box_safety_in(const OSolid *s, const double *p) {
  double m = fabs(p[0]) - s->a, d;
  d = fabs(p[1]) - s->b; if (d > m) m = d;
  d = fabs(p[2]) - s->c; if (d > m) m = d;
  return m > 0.0 ? m : 0.0;
}

static double box_safety_out(const OSolid *s, const double *p) {
  double m = s->a - fabs(p[0]), d;
  d = s->b - fabs(p[1]); if (d < m) m = d;
  d = s->c - fabs(p[2]); if (d < m) m = d;
  return m > 0.0 ? m : 0.0;
}

static int orb_inside(const OSolid *s, const double *p, const double *v) {
  double r2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
  double ro = s->a + kHalf, ri = s->a - kHalf;
  if (r2 > ro * ro) return 0;
  if (r2 < ri * ri) return 1;
  return p[0] * v[0] + p[1] * v[1] + p[2] * v[2] < 0.0;
}

/* Roots of t^2 + 2 b t + c = 0 computed without cancellation.  Returns 0 if
 * the discriminant is not positive. */
static int sphere_roots(double b, double c, double *lo, double *hi) {
  double disc = b * b - c;
  if (!(disc > 0.0)) return 0;
  double sq = sqrt(disc);
  double q = b >= 0.0 ? -(b + sq) : -(b - sq);
  double r1 = q, r2 = c / q;
  *lo = r1 < r2 ? r1 : r2;
  *hi = r1 < r2 ? r2 : r1;
  return 1;
}

static double orb_dist_in(const OSolid *s, const double *p, const double *v) {
  double b = p[0] * v[0] + p[1] * v[1] + p[2] * v[2];
  double c = p[0] * p[0] + p[1] * p[1] + p[2] * p[2] - s->a * s->a;
  double lo, hi;
  if (!sphere_roots(b, c, &lo, &hi)) return O_INF;
  return lo > kHalf ? lo : O_INF;
}

static double orb_dist_out(const OSolid *s, const double *p, const double *v) {
  double b = p[0] * v[0] + p[1] * v[1] + p[2] * v[2];
  double c = p[0] * p[0] + p[1] * p[1] + p[2] * p[2] - s->a * s->a;
  double lo, hi;
  if (!sphere_roots(b, c, &lo, &hi)) return 0.0;
  return hi > 0.0 ? hi : 0.0;
}

static double orb_safety_in(const OSolid *s, const double *p) {
  double d = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]) - s->a;
  return d > 0.0 ? d : 0.0;
}

static double orb_safety_out(const OSolid *s, const double *p) {
  double d = s->a - sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
  return d > 0.0 ? d : 0.0;
}

/* Tube segment.  phi_s(p) = cross(u_start, p) and phi_e(p) = cross(p, u_end)
 * are the signed distances to the lines through the start and end half-planes,
 * positive on the solid's side.  For dphi <= pi the phi range is the
 * intersection of the two half-planes, for dphi > pi their union. */
static double phi_s(const OSolid *s, double x, double y) { return s->cs * y - s->ss * x; }
static double phi_e(const OSolid *s, double x, double y) { return s->se * x - s->ce * y; }

static int phi_within(const OSolid *s, double x, double y, double tol) {
  if (!s->seg) return 1;
  double a = phi_s(s, x, y), b = phi_e(s, x, y);
  return s->wide ? (a >= -tol || b >= -tol) : (a >= -tol && b >= -tol);
}

static int tube_inside(const OSolid *s, const double *p, const double *v) {
  const double x = p[0], y = p[1], z = p[2];
  const double rmin = s->a, rmax = s->b, hz = s->c;
  double r2 = x * x + y * y;
  double sz = fabs(z) - hz;
  if (sz > kHalf) return 0;
  double ro = rmax + kHalf, rmi = rmax - kHalf;
  if (r2 > ro * ro) return 0;
  int nz = sz >= -kHalf;
  int nrmax = r2 >= rmi * rmi;
  int nrmin = 0;
  if (rmin > 0.0) {
    double ri = rmin - kHalf, rio = rmin + kHalf;
    if (r2 < ri * ri) return 0;
    nrmin = r2 <= rio * rio;
  }
  int ns = 0, ne = 0;
  if (s->seg) {
    double a = phi_s(s, x, y), b = phi_e(s, x, y);
    if (!s->wide) {
      if (a < -kHalf || b < -kHalf) return 0;
      ns = a <= kHalf;
      ne = b <= kHalf;
    } else {
      double m = a >= b ? a : b;
      if (m < -kHalf) return 0;
      if (m <= kHalf) { if (a >= b) ns = 1; else ne = 1; }
    }
  }
  if (!(nz || nrmax || nrmin || ns || ne)) return 1;
  double vr = x * v[0] + y * v[1];
  if (nz && !(z * v[2] < 0.0)) return 0;
  if (nrmax && !(vr < 0.0)) return 0;
  if (nrmin && !(vr > 0.0)) return 0;
  if (ns && !(s->ss * v[0] - s->cs * v[1] < 0.0)) return 0;
  if (ne && !(-s->se * v[0] + s->ce * v[1] < 0.0)) return 0;
  return 1;
}

/* Hit-point checks: the point of a candidate intersection must lie on the
 * solid's boundary, every other constraint widened by kHalf. */
static int tube_hit_r_ok(const OSolid *s, double x, double y) {
  double r2 = x * x + y * y, ro = s->b + kHalf;
  if (r2 > ro * ro) return 0;
  if (s->a > 0.0) { double ri = s->a - kHalf; if (r2 < ri * ri) return 0; }
  return 1;
}

/* Roots of a t^2 + 2 b t + c = 0 (a > 0) without cancellation. */
static int cyl_roots(double a, double b, double c, double *lo, double *hi) {
  double disc = b * b - a * c;
  if (!(disc > 0.0)) return 0;
  double sq = sqrt(disc);
  double q = b >= 0.0 ? -(b + sq) : -(b - sq);
  double r1 = q / a, r2 = c / q;
  *lo = r1 < r2 ? r1 : r2;
  *hi = r1 < r2 ? r2 : r1;
  return 1;
}

/* mode = +1: entering intersections with t > kHalf (DistanceToIn);
 * mode = -1: exiting intersections with t > -kHalf (DistanceToOut). */
static double tube_cross(const OSolid *s, const double *p, const double *v, int mode) {
  const double x = p[0], y = p[1], z = p[2];
  const double rmin = s->a, rmax = s->b, hz = s->c;
  const double tmin = mode > 0 ? kHalf : -kHalf;
  double best = O_INF;
  /* z planes: outward normal (0, 0, sigma); entering iff sigma * vz < 0. */
  if (v[2] != 0.0) {
    for (int k = 0; k < 2; ++k) {
      double sg = k == 0 ? 1.0 : -1.0;
      int entering = sg * v[2] < 0.0;
      if ((mode > 0) != entering) continue;
      double t = (sg * hz - z) / v[2];
      if (!(t > tmin && t < best)) continue;
      double qx = x + t * v[0], qy = y + t * v[1];
      if (tube_hit_r_ok(s, qx, qy) && phi_within(s, qx, qy, kHalf)) best = t;
    }
  }
  double a = v[0] * v[0] + v[1] * v[1];
  if (a > 0.0) {
    double b = x * v[0] + y * v[1];
    double r2 = x * x + y * y;
    double lo, hi;
    /* outer cylinder: the solid is inside it; enter at the low root, exit at the high root. */
    if (cyl_roots(a, b, r2 - rmax * rmax, &lo, &hi)) {
      double t = mode > 0 ? lo : hi;
      if (t > tmin && t < best) {
        double qz = z + t * v[2];
        if (fabs(qz) <= hz + kHalf && phi_within(s, x + t * v[0], y + t * v[1], kHalf)) best = t;
      }
    }
    /* inner cylinder: the solid is outside it; enter the solid at the high root, leave at the low root. */
    if (rmin > 0.0 && cyl_roots(a, b, r2 - rmin * rmin, &lo, &hi)) {
      double t = mode > 0 ? hi : lo;
      if (t > tmin && t < best) {
        double qz = z + t * v[2];
        if (fabs(qz) <= hz + kHalf && phi_within(s, x + t * v[0], y + t * v[1], kHalf)) best = t;
      }
    }
  }
  if (s->seg) {
    /* start half-plane: outward normal (ss, -cs); dn = v . n */
    double dn = s->ss * v[0] - s->cs * v[1];
    if (dn != 0.0 && ((mode > 0) == (dn < 0.0))) {
      double t = phi_s(s, x, y) / dn;
      if (t > tmin && t < best) {
        double qx = x + t * v[0], qy = y + t * v[1], qz = z + t * v[2];
        if (s->cs * qx + s->ss * qy >= -kHalf && tube_hit_r_ok(s, qx, qy) && fabs(qz) <= hz + kHalf) best = t;
      }
    }
    /* end half-plane: outward normal (-se, ce) */
    double de = -s->se * v[0] + s->ce * v[1];
    if (de != 0.0 && ((mode > 0) == (de < 0.0))) {
      double t = phi_e(s, x, y) / de;
      if (t > tmin && t < best) {
        double qx = x + t * v[0], qy = y + t * v[1], qz = z + t * v[2];
        if (s->ce * qx + s->se * qy >= -kHalf && tube_hit_r_ok(s, qx, qy) && fabs(qz) <= hz + kHalf) best = t;
      }
    }
  }
  return best;
}

static double tube_dist_in(const OSolid *s, const double *p, const double *v) { return tube_cross(s, p, v, +1); }

static double tube_dist_out(const OSolid *s, const double *p, const double *v) {
  double t = tube_cross(s, p, v, -1);
  if (t == O_INF) return 0.0;
  return t > 0.0 ? t : 0.0;
}

static double tube_safety_in(const OSolid *s, const double *p) {
  double r = sqrt(p[0] * p[0] + p[1] * p[1]);
  double m = r - s->b, d;
  if (s->a > 0.0) { d = s->a - r; if (d > m) m = d; }
  d = fabs(p[2]) - s->c; if (d > m) m = d;
  if (s->seg) {
    double a = -phi_s(s, p[0], p[1]), b = -phi_e(s, p[0], p[1]);
    d = s->wide ? (a < b ? a : b) : (a > b ? a : b);
    if (d > m) m = d;
  }
  return m > 0.0 ? m : 0.0;
}

static double tube_safety_out(const OSolid *s, const double *p) {
  double r = sqrt(p[0] * p[0] + p[1] * p[1]);
  double m = s->b - r, d;
  if (s->a > 0.0) { d = r - s->a; if (d < m) m = d; }
  d = s->c - fabs(p[2]); if (d < m) m = d;
  if (s->seg) {
    d = fabs(phi_s(s, p[0], p[1])); if (d < m) m = d;
    d = fabs(phi_e(s, p[0], p[1])); if (d < m) m = d;
  }
  return m > 0.0 ? m : 0.0;
}

/* Cone, full in phi.  Between z = -hz and +hz the solid is Rin(z) <= r <= Rout(z) with
 * Rout(z) = ko z + co and Rin(z) = ki z + ci (Rin = 0: no inner surface).  The band of a
 * conical surface is measured along r at the point's z.  Outward normal of the outer surface
 * along (x / r, y / r, -ko); of the inner surface (the solid lies outside it) along
 * (-x / r, -y / r, ki).  The end faces' radii are R(+-hz) evaluated the same way. */
static double cone_r(double k, double c, double z) { return k * z + c; }

static int cone_inside(const OSolid *s, const double *p, const double *v) {
  const double x = p[0], y = p[1], z = p[2], hz = s->c;
  double sz = fabs(z) - hz;
  if (sz > kHalf) return 0;
  double r2 = x * x + y * y;
  double ro = cone_r(s->ko, s->co, z);
  double rop = ro + kHalf, rom = ro - kHalf;
  if (r2 > rop * rop) return 0;
  int nz = sz >= -kHalf;
  int nrmax = r2 >= rom * rom;
  int nrmin = 0;
  if (s->has_in) {
    double ri = cone_r(s->ki, s->ci, z);
    double rim = ri - kHalf, rip = ri + kHalf;
    if (r2 < rim * rim) return 0;
    nrmin = r2 <= rip * rip;
  }
  if (!(nz || nrmax || nrmin)) return 1;
  double r = sqrt(r2);
  double vr = x * v[0] + y * v[1];
  if (nz && !(z * v[2] < 0.0)) return 0;
  if (nrmax && !(vr - s->ko * r * v[2] < 0.0)) return 0;
  if (nrmin && !(vr - s->ki * r * v[2] > 0.0)) return 0;
  return 1;
}

/* mode = +1: entering crossings with t > kHalf; mode = -1: exiting crossings with t > -kHalf. */
static double cone_cross(const OSolid *s, const double *p, const double *v, int mode) {
  const double x = p[0], y = p[1], z = p[2], hz = s->c;
  const double tmin = mode > 0 ? kHalf : -kHalf;
  double best = O_INF;
  /* end faces: the hit radius between the inner and outer radius of that end */
  if (v[2] != 0.0) {
    for (int k = 0; k < 2; ++k) {
      double sg = k == 0 ? 1.0 : -1.0;
      int entering = sg * v[2] < 0.0;
      if ((mode > 0) != entering) continue;
      double t = (sg * hz - z) / v[2];
      if (!(t > tmin && t < best)) continue;
      double qx = x + t * v[0], qy = y + t * v[1];
      double r2 = qx * qx + qy * qy;
      double ro = cone_r(s->ko, s->co, sg * hz) + kHalf;
      if (r2 > ro * ro) continue;
      if (s->has_in) {
        double ri = cone_r(s->ki, s->ci, sg * hz) - kHalf;
        if (r2 < ri * ri) continue;
      }
      best = t;
    }
  }
  /* conical surfaces: (x + t vx)^2 + (y + t vy)^2 = (k (z + t vz) + c)^2, i.e.
   * a t^2 + 2 b t + cc = 0; d = a t + b is half the rate of change of r^2 - R^2 */
  for (int w = 0; w < 1 + s->has_in; ++w) {
    const double k = w == 0 ? s->ko : s->ki, c = w == 0 ? s->co : s->ci;
    const double rz = cone_r(k, c, z);
    const double a = v[0] * v[0] + v[1] * v[1] - k * k * v[2] * v[2];
    const double b = x * v[0] + y * v[1] - k * v[2] * rz;
    const double cc = x * x + y * y - rz * rz;
    double roots[2];
    int nr = 0;
    if (a != 0.0) {
      double disc = b * b - a * cc;
      if (disc > 0.0) {
        double sq = sqrt(disc);
        double q = b >= 0.0 ? -(b + sq) : -(b - sq);
        roots[nr++] = q / a;
        roots[nr++] = cc / q;
      }
    } else if (b != 0.0) {
      roots[nr++] = -cc / (2.0 * b);
    }
    for (int i = 0; i < nr; ++i) {
      const double t = roots[i];
      if (!(t > tmin && t < best)) continue;
      const double d = a * t + b;
      /* into the solid: through the outer surface r^2 - R^2 decreases, through the inner one it grows */
      const int entering = w == 0 ? d < 0.0 : d > 0.0;
      if ((mode > 0) != entering) continue;
      const double qz = z + t * v[2];
      if (fabs(qz) > hz + kHalf) continue;
      if (!(cone_r(k, c, qz) >= 0.0)) continue;   /* the other half of the double cone */
      best = t;
    }
  }
  return best;
}

static double cone_dist_in(const OSolid *s, const double *p, const double *v) { return cone_cross(s, p, v, +1); }

static double cone_dist_out(const OSolid *s, const double *p, const double *v) {
  double t = cone_cross(s, p, v, -1);
  if (t == O_INF) return 0.0;
  return t > 0.0 ? t : 0.0;
}

/* Safety: perpendicular distances (in the meridian plane) to the lines of the conical surfaces,
 * which bound the distances to the surfaces from below, and the distance to the end planes. */
static double cone_safety_in(const OSolid *s, const double *p) {
  double r = sqrt(p[0] * p[0] + p[1] * p[1]);
  double m = fabs(p[2]) - s->c, d;
  d = (r - cone_r(s->ko, s->co, p[2])) * s->cao; if (d > m) m = d;
  if (s->has_in) { d = (cone_r(s->ki, s->ci, p[2]) - r) * s->cai; if (d > m) m = d; }
  return m > 0.0 ? m : 0.0;
}

static double cone_safety_out(const OSolid *s, const double *p) {
  double r = sqrt(p[0] * p[0] + p[1] * p[1]);
  double m = s->c - fabs(p[2]), d;
  d = (cone_r(s->ko, s->co, p[2]) - r) * s->cao; if (d < m) m = d;
  if (s->has_in) { d = (r - cone_r(s->ki, s->ci, p[2])) * s->cai; if (d < m) m = d; }
  return m > 0.0 ? m : 0.0;
}

/* "Fork" dispatch on the solid type (the paper's replacement for virtual calls, Sec. 3.3). */
static int s_inside(const OSolid *s, const double *p, const double *v) {
  switch (s->kind) {
    case O_BOX: return box_inside(s, p, v);
    case O_TUBE: return tube_inside(s, p, v);
    case O_CONE: return cone_inside(s, p, v);
    default: return orb_inside(s, p, v);
  }
}
static double s_dist_in(const OSolid *s, const double *p, const double *v) {
  switch (s->kind) {
    case O_BOX: return box_dist_in(s, p, v);
    case O_TUBE: return tube_dist_in(s, p, v);
    case O_CONE: return cone_dist_in(s, p, v);
    default: return orb_dist_in(s, p, v);
  }
}
static double s_dist_out(const OSolid *s, const double *p, const double *v) {
  switch (s->kind) {
    case O_BOX: return box_dist_out(s, p, v);
    case O_TUBE: return tube_dist_out(s, p, v);
    case O_CONE: return cone_dist_out(s, p, v);
    default: return orb_dist_out(s, p, v);
  }
}
static double s_safety_in(const OSolid *s, const double *p) {
  switch (s->kind) {
    case O_BOX: return box_safety_in(s, p);
    case O_TUBE: return tube_safety_in(s, p);
    case O_CONE: return cone_safety_in(s, p);
    default: return orb_safety_in(s, p);
  }
}
static double s_safety_out(const OSolid *s, const double *p) {
  switch (s->kind) {
    case O_BOX: return box_safety_out(s, p);
    case O_TUBE: return tube_safety_out(s, p);
    case O_CONE: return cone_safety_out(s, p);
    default: return orb_safety_out(s, p);
  }
}

/* Solid-level entry points (local frame) for the closed-form pins. */
int o_solid_inside(int gi, int solid, const double *p, const double *v) { return s_inside(&G[gi]->sol[solid], p, v); }
double o_solid_dist_in(int gi, int solid, const double *p, const double *v) { return s_dist_in(&G[gi]->sol[solid], p, v); }
double o_solid_dist_out(int gi, int solid, const double *p, const double *v) { return s_dist_out(&G[gi]->sol[solid], p, v); }
double o_solid_safety_in(int gi, int solid, const double *p) { return s_safety_in(&G[gi]->sol[solid], p); }
double o_solid_safety_out(int gi, int solid, const double *p) { return s_safety_out(&G[gi]->sol[solid], p); }

/* ------------------------------------------------------------------ navigation */

/* Point and direction in the frame of path[depth-1], applying each level's placement from the world down. */
static void frame_of(const OGeom *g, const int *path, int depth, const double *p, const double *v, double *pl, double *vl) {
  double pa[3] = {p[0], p[1], p[2]}, va[3] = {v[0], v[1], v[2]};
  for (int k = 0; k < depth; ++k) {
    to_local(&g->vol[path[k]], pa, va, pl, vl);
    memcpy(pa, pl, sizeof(pa));
    memcpy(va, vl, sizeof(va));
  }
  memcpy(pl, pa, sizeof(pa));
  memcpy(vl, va, sizeof(va));
}

/* ------------------------------------------------------------------ uniform-grid acceleration
 * Timing mode only (the CPU baseline of the benchmark): the plain definitions above search every
 * daughter; with o_build_grids() a mother with at least O_GRID_MIN daughters gets a uniform grid over
 * its bounding box, and
 *  - locate tests only the daughters listed in the point's cell, in placement order (a daughter that
 *    contains the point, band included, overlaps the cell: lists are built from bounding boxes grown
 *    by O_GRID_PAD, far above the tolerance band and every rounding error of the cell lookup);
 *  - the step visits the cells along the ray (3-D DDA) from the point's cell until the next cell
 *    begins beyond the best distance found, evaluating each listed daughter once; a daughter entered
 *    at t <= best has its entry point in a cell that begins at or before t, so it is evaluated; among
 *    equal distances the lower placement index wins, as in the brute-force loop.
 * The results are those of the brute-force search (tests compare histories on subsets of every
 * workload).  Written independently of the library's voxels. */
#define O_GRID_MIN 8
#define O_GRID_PAD 1e-6
#define O_GRID_MAXN 128
#define O_GRID_SEEN 512

/* Half-extents of a solid's bounding box in its own frame (tubes and cones: the full cylinder). */
static void solid_half(const OSolid *s, double *h) {
  if (s->kind == O_BOX) { h[0] = s->a; h[1] = s->b; h[2] = s->c; }
  else if (s->kind == O_ORB) { h[0] = h[1] = h[2] = s->a; }
  else if (s->kind == O_TUBE) { h[0] = h[1] = s->b; h[2] = s->c; }
  else {
    double r = fmax(fabs(s->ko * s->c + s->co), fabs(-s->ko * s->c + s->co));
    h[0] = h[1] = r; h[2] = s->c;
  }
}

static void build_grid(OGeom *g, int m) {
  const OVol *mv = &g->vol[m];
  double H[3];
  solid_half(&g->sol[mv->solid], H);
  double dlo[3], dhi[3], mean[3] = {0, 0, 0};
  double (*bl)[3] = (double (*)[3])malloc((size_t)mv->ndau * sizeof(double[3]));
  double (*bh)[3] = (double (*)[3])malloc((size_t)mv->ndau * sizeof(double[3]));
  for (int k = 0; k < mv->ndau; ++k) {
    const OVol *d = &g->vol[g->dau[mv->first + k]];
    double h[3];
    solid_half(&g->sol[d->solid], h);
    const double ex = fabs(d->c) * h[0] + fabs(d->s) * h[1], ey = fabs(d->s) * h[0] + fabs(d->c) * h[1];
    const double e[3] = {ex, ey, h[2]};
    for (int a = 0; a < 3; ++a) {
      bl[k][a] = d->t[a] - e[a] - O_GRID_PAD;
      bh[k][a] = d->t[a] + e[a] + O_GRID_PAD;
      mean[a] += 2.0 * e[a] / mv->ndau;
    }
  }
  OGrid *gr = (OGrid *)calloc(1, sizeof(OGrid));
  long ncell = 1;
  for (int a = 0; a < 3; ++a) {
    dlo[a] = -H[a];
    dhi[a] = H[a];
    int n = (int)ceil(2.0 * H[a] / fmax(mean[a], 1e-9));
    n = n < 1 ? 1 : (n > O_GRID_MAXN ? O_GRID_MAXN : n);
    gr->n[a] = n;
    gr->lo[a] = dlo[a];
    gr->w[a] = (dhi[a] - dlo[a]) / n;
    ncell *= n;
  }
  /* counting pass, then fill (daughters in placement order) */
  gr->off = (int *)calloc((size_t)ncell + 1, sizeof(int));
  int lo3[3], hi3[3];
  for (int pass = 0; pass < 2; ++pass) {
    int *fill = pass ? (int *)calloc((size_t)ncell, sizeof(int)) : NULL;
    for (int k = 0; k < mv->ndau; ++k) {
      for (int a = 0; a < 3; ++a) {
        lo3[a] = (int)floor((bl[k][a] - gr->lo[a]) / gr->w[a]);
        hi3[a] = (int)floor((bh[k][a] - gr->lo[a]) / gr->w[a]);
        lo3[a] = lo3[a] < 0 ? 0 : (lo3[a] >= gr->n[a] ? gr->n[a] - 1 : lo3[a]);
        hi3[a] = hi3[a] < 0 ? 0 : (hi3[a] >= gr->n[a] ? gr->n[a] - 1 : hi3[a]);
      }
      for (int i = lo3[0]; i <= hi3[0]; ++i)
        for (int j = lo3[1]; j <= hi3[1]; ++j)
          for (int l = lo3[2]; l <= hi3[2]; ++l) {
            const long c = ((long)i * gr->n[1] + j) * gr->n[2] + l;
            if (pass == 0) gr->off[c + 1]++;
            else gr->lst[gr->off[c] + fill[c]++] = g->dau[mv->first + k];
          }
    }
    if (pass == 0) {
      for (long c = 0; c < ncell; ++c) gr->off[c + 1] += gr->off[c];
      gr->lst = (int *)malloc((size_t)(gr->off[ncell] > 0 ? gr->off[ncell] : 1) * sizeof(int));
    } else {
      free(fill);
    }
  }
  free(bl);
  free(bh);
  g->grid[m] = gr;
}

/* Build the grids of every mother with at least O_GRID_MIN daughters and switch the timing mode on
 * (on = 0 switches it off again; the grids are kept). */
void o_use_grids(int gi, int on) {
  OGeom *g = G[gi];
  if (on && !g->grid) {
    g->grid = (OGrid **)calloc((size_t)g->nvol, sizeof(OGrid *));
    for (int m = 0; m < g->nvol; ++m)
      if (g->vol[m].ndau >= O_GRID_MIN) build_grid(g, m);
  }
  g->use_grid = on;
}

static int grid_cell(const OGrid *gr, const double *p, int *c) {
  for (int a = 0; a < 3; ++a) {
    int k = (int)floor((p[a] - gr->lo[a]) / gr->w[a]);
    c[a] = k < 0 ? 0 : (k >= gr->n[a] ? gr->n[a] - 1 : k);
  }
  return (c[0] * gr->n[1] + c[1]) * gr->n[2] + c[2];
}

static const OGrid *grid_of(const OGeom *g, int m) {
  return (g->use_grid && g->grid) ? g->grid[m] : NULL;
}

static uint64_t *g_cnt_inside = NULL;   /* optional per-call counter of Inside tests */

/* Enter, repeatedly, the first daughter in placement order whose solid contains the point. */
static void descend(const OGeom *g, int *path, int *depth, double *pl, double *vl, uint64_t *cnt) {
  for (;;) {
    const OVol *m = &g->vol[path[*depth - 1]];
    int found = -1;
    double dl[3], dv[3];
    /* the daughters to test, in placement order: all of them, or those of the point's grid cell */
    const int *ds = g->dau + m->first;
    int nd = m->ndau;
    const OGrid *gr = grid_of(g, path[*depth - 1]);
    if (gr) {
      int c[3];
      const int cell = grid_cell(gr, pl, c);
      ds = gr->lst + gr->off[cell];
      nd = gr->off[cell + 1] - gr->off[cell];
    }
    for (int k = 0; k < nd; ++k) {
      int d = ds[k];
      to_local(&g->vol[d], pl, vl, dl, dv);
      if (cnt) cnt[C_INSIDE]++;
      if (s_inside(&g->sol[g->vol[d].solid], dl, dv)) { found = d; break; }
    }
    if (found < 0 || *depth >= O_DMAX) return;
    path[(*depth)++] = found;
    memcpy(pl, dl, 3 * sizeof(double));
    memcpy(vl, dv, 3 * sizeof(double));
  }
}

static int locate_impl(const OGeom *g, const double *p, const double *v, int *path, uint64_t *cnt) {
  double pl[3], vl[3];
  to_local(&g->vol[0], p, v, pl, vl);
  if (cnt) cnt[C_INSIDE]++;
  if (!s_inside(&g->sol[g->vol[0].solid], pl, vl)) return 0;
  int depth = 1;
  path[0] = 0;
  descend(g, path, &depth, pl, vl, cnt);
  return depth;
}

/* Navigation problem 1 (Sec. 3.2): which volumes contain the point.  Returns
 * the depth (0 = outside the world) and writes path[0..depth). */
int o_locate(int gi, const double *p, const double *v, int *path) {
  for (int k = 0; k < O_DMAX; ++k) path[k] = -1;
  return locate_impl(G[gi], p, v, path, NULL);
}

/* After a move: leave every level whose solid no longer contains the point
 * (direction aware), then descend from the deepest level that does. */
static int relocate_impl(const OGeom *g, int *path, int depth, const double *p, const double *v, uint64_t *cnt) {
  double pl[3], vl[3];
  while (depth > 0) {
    frame_of(g, path, depth, p, v, pl, vl);
    if (cnt) cnt[C_INSIDE]++;
    if (s_inside(&g->sol[g->vol[path[depth - 1]].solid], pl, vl)) break;
    path[--depth] = -1;
  }
  if (depth == 0) return 0;
  descend(g, path, &depth, pl, vl, cnt);
  return depth;
}

int o_relocate(int gi, int *path, int depth, const double *p, const double *v) {
  return relocate_impl(G[gi], path, depth, p, v, NULL);
}

/* Navigation problem 2 (Sec. 3.2): the geometric step from p along v inside
 * path[depth-1].  Minimum of the volume's DistanceToOut (limiter -1) and every
 * daughter's DistanceToIn (limiter = daughter id).  Ties: a daughter beats the
 * mother; between daughters the lower placement index wins.  Brute-force
 * isotropic safety.  Returns the geometric step. */
/* The step of the timing mode: the cells along the ray, each listed daughter once (see above).
 * Returns 0 when more daughters were met than it can remember (the caller then searches them all). */
static int grid_step(const OGeom *g, const OGrid *gr, const double *pl, const double *vl, double *best_io,
                     int *lim_io, uint64_t *cnt) {
  int c[3], st[3];
  double tmax[3], tdel[3];
  grid_cell(gr, pl, c);
  for (int a = 0; a < 3; ++a) {
    if (vl[a] > 0.0) {
      st[a] = 1;
      tmax[a] = (gr->lo[a] + (c[a] + 1) * gr->w[a] - pl[a]) / vl[a];
      tdel[a] = gr->w[a] / vl[a];
    } else if (vl[a] < 0.0) {
      st[a] = -1;
      tmax[a] = (gr->lo[a] + c[a] * gr->w[a] - pl[a]) / vl[a];
      tdel[a] = -gr->w[a] / vl[a];
    } else {
      st[a] = 0;
      tmax[a] = O_INF;
      tdel[a] = O_INF;
    }
  }
  int seen[O_GRID_SEEN], nseen = 0;
  double best = *best_io;
  int lim = *lim_io;
  for (;;) {
    const int cell = (c[0] * gr->n[1] + c[1]) * gr->n[2] + c[2];
    for (int k = gr->off[cell]; k < gr->off[cell + 1]; ++k) {
      const int d = gr->lst[k];
      int dup = 0;
      for (int q = 0; q < nseen; ++q)
        if (seen[q] == d) { dup = 1; break; }
      if (dup) continue;
      if (nseen == O_GRID_SEEN) return 0;
      seen[nseen++] = d;
      double dl[3], dv[3];
      to_local(&g->vol[d], pl, vl, dl, dv);
      if (cnt) cnt[C_DIST_IN]++;
      const double t = s_dist_in(&g->sol[g->vol[d].solid], dl, dv);
      if (t < O_INF && (t < best || (t == best && (lim == LIM_MOTHER || d < lim)))) { best = t; lim = d; }
    }
    const int a = tmax[0] <= tmax[1] ? (tmax[0] <= tmax[2] ? 0 : 2) : (tmax[1] <= tmax[2] ? 1 : 2);
    if (!(tmax[a] <= best)) break;   /* the next cell begins beyond the best distance */
    c[a] += st[a];
    if (st[a] == 0 || c[a] < 0 || c[a] >= gr->n[a]) break;
    tmax[a] += tdel[a];
  }
  *best_io = best;
  *lim_io = lim;
  return 1;
}

static double geom_step(const OGeom *g, const int *path, int depth, const double *p, const double *v,
                        int *limiter, double *safety, uint64_t *cnt) {
  double pl[3], vl[3];
  frame_of(g, path, depth, p, v, pl, vl);
  const OVol *m = &g->vol[path[depth - 1]];
  const OSolid *ms = &g->sol[m->solid];
  double best = s_dist_out(ms, pl, vl);
  int lim = LIM_MOTHER;
  const OGrid *gr = safety ? NULL : grid_of(g, path[depth - 1]);
  if (gr) {
    double b = best;
    int l = lim;
    if (grid_step(g, gr, pl, vl, &b, &l, cnt)) {
      *limiter = l;
      return b;
    }
  }
  double saf = safety ? s_safety_out(ms, pl) : 0.0;
  for (int k = 0; k < m->ndau; ++k) {
    int d = g->dau[m->first + k];
    double dl[3], dv[3];
    to_local(&g->vol[d], pl, vl, dl, dv);
    const OSolid *ds = &g->sol[g->vol[d].solid];
    if (cnt) cnt[C_DIST_IN]++;
    double t = s_dist_in(ds, dl, dv);
    if (t < O_INF && (t < best || (t == best && lim == LIM_MOTHER))) { best = t; lim = d; }
    if (safety) { double sd = s_safety_in(ds, dl); if (sd < saf) saf = sd; }
  }
  *limiter = lim;
  if (safety) *safety = saf;
  return best;
}

/* compute_step with a proposed physics step: the physics step wins only if strictly shorter.
 * out_safety may be NULL (no safety: the timing mode's grids may then serve the step). */
int o_compute_step(int gi, int depth, const int *path, const double *p, const double *v, double proposed,
                   double *out_step, int *out_limiter, double *out_safety) {
  const OGeom *g = G[gi];
  if (depth <= 0) return -1;
  int lim;
  double saf = 0.0;
  double s = geom_step(g, path, depth, p, v, &lim, out_safety ? &saf : NULL, NULL);
  if (proposed < s) { s = proposed; lim = LIM_PHYS; }
  *out_step = s;
  *out_limiter = lim;
  if (out_safety) *out_safety = saf;
  return 0;
}

/* ------------------------------------------------------------------ random numbers */

static void philox_round(uint32_t *c, const uint32_t *k) {
  uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
  uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
  uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  uint32_t o0 = hi1 ^ c[1] ^ k[0], o1 = lo1, o2 = hi0 ^ c[3] ^ k[1], o3 = lo0;
  c[0] = o0; c[1] = o1; c[2] = o2; c[3] = o3;
}

/* Philox4x32 with 10 rounds: S-box rounds with the key bumped by the Weyl
 * constants (0x9E3779B9, 0xBB67AE85) between rounds. */
void o_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k[0] += 0x9E3779B9u; k[1] += 0xBB67AE85u; }
    philox_round(c, k);
  }
  memcpy(out, c, sizeof(c));
}

typedef struct { uint64_t seed; int64_t tid; uint32_t stream, draw; } ORng;

/* Two uniforms in (0, 1] from one block: the top 53 bits of (x1:x0) and of (x3:x2), each
 * plus one, times 2^-53.  A draw site takes whole blocks: a single uniform uses the first. */
static void rng_pair(ORng *r, double *ua, double *ub) {
  uint32_t ctr[4] = {r->draw++, (uint32_t)(uint64_t)r->tid, (uint32_t)((uint64_t)r->tid >> 32), r->stream};
  uint32_t key[2] = {(uint32_t)r->seed, (uint32_t)(r->seed >> 32)};
  uint32_t x[4];
  o_philox4x32_10(ctr, key, x);
  uint64_t wa = ((uint64_t)x[1] << 32) | x[0];
  uint64_t wb = ((uint64_t)x[3] << 32) | x[2];
  *ua = (double)((wa >> 11) + 1) * 0x1.0p-53;
  *ub = (double)((wb >> 11) + 1) * 0x1.0p-53;
}

static double rng_u(ORng *r) {
  double a, b;
  rng_pair(r, &a, &b);
  return a;
}

double o_uniform(uint64_t seed, int64_t tid, uint32_t stream, uint32_t draw) {
  ORng r = {seed, tid, stream, draw};
  return rng_u(&r);
}

void o_uniform_pair(uint64_t seed, int64_t tid, uint32_t stream, uint32_t draw, double *out) {
  ORng r = {seed, tid, stream, draw};
  rng_pair(&r, &out[0], &out[1]);
}

/* FNV-1a, 64 bit, over little-endian bytes. */
#define FNV_OFFSET 0xcbf29ce484222325ull
#define FNV_PRIME 0x100000001b3ull
uint64_t o_fnv1a(const uint8_t *bytes, int64_t n) {
  uint64_t h = FNV_OFFSET;
  for (int64_t i = 0; i < n; ++i) { h ^= bytes[i]; h *= FNV_PRIME; }
  return h;
}

static uint64_t hash_step(uint64_t h, int32_t leaf, int32_t limiter, int32_t event) {
  int32_t w[3] = {leaf, limiter, event};
  for (int k = 0; k < 3; ++k) {
    uint32_t u = (uint32_t)w[k];
    for (int b = 0; b < 4; ++b) { h ^= (u >> (8 * b)) & 0xffu; h *= FNV_PRIME; }
  }
  return h;
}

/* ------------------------------------------------------------------ physics */

#define ME_C2 0.51099895

/* Linear attenuation coefficients at energy E: binary search for E_k <= E < E_{k+1},
 * then lin-lin interpolation; clamped to the table ends. */
static void mu_lookup(const OMat *m, double E, double *mu_tot, double *mu_pe) {
  int n = m->n;
  double mc, mp;
  if (E <= m->E[0]) { mc = m->muC[0]; mp = m->muP[0]; }
  else if (E >= m->E[n - 1]) { mc = m->muC[n - 1]; mp = m->muP[n - 1]; }
  else {
    int lo = 0, hi = n - 1;
    while (hi - lo > 1) { int mid = (lo + hi) / 2; if (m->E[mid] <= E) lo = mid; else hi = mid; }
    double f = (E - m->E[lo]) / (m->E[lo + 1] - m->E[lo]);
    mc = m->muC[lo] + f * (m->muC[lo + 1] - m->muC[lo]);
    mp = m->muP[lo] + f * (m->muP[lo + 1] - m->muP[lo]);
  }
  *mu_tot = mc + mp;
  *mu_pe = mp;
}

void o_mu(int gi, int mat, double E, double *out) {
  double t, p;
  mu_lookup(&G[gi]->mat[mat], E, &t, &p);
  out[0] = t; out[1] = p;
}

/* Kahn's rejection method for the Klein-Nishina distribution of eta = E / E'
 * (three uniforms per trial: r1, r2 from one block, r3 from the next).  Returns the
 * number of trials (0 = cap hit). */
static int kahn(double E, ORng *r, double *eta_out, double *cost_out) {
  double al = E / ME_C2;
  double p1 = (1.0 + 2.0 * al) / (9.0 + 2.0 * al);
  for (int trial = 1; trial <= 1000; ++trial) {
    double r1, r2, r3, unused;
    rng_pair(r, &r1, &r2);
    rng_pair(r, &r3, &unused);
    double eta, cost;
    if (r1 <= p1) {
      eta = 1.0 + 2.0 * al * r2;
      if (!(r3 <= 4.0 * (1.0 / eta - 1.0 / (eta * eta)))) continue;
      cost = 1.0 - (eta - 1.0) / al;
    } else {
      eta = (1.0 + 2.0 * al) / (1.0 + 2.0 * al * r2);
      cost = 1.0 - (eta - 1.0) / al;
      if (!(r3 <= 0.5 * (cost * cost + 1.0 / eta))) continue;
    }
    *eta_out = eta;
    *cost_out = cost;
    return trial;
  }
  *eta_out = 1.0;
  *cost_out = 1.0;
  return 0;
}

/* Uniform azimuth by rejection on the unit disc: (cos 2psi, sin 2psi) of a uniform point
 * (one block per trial). */
static int azimuth(ORng *r, double *cph, double *sph) {
  for (int trial = 1; trial <= 1000; ++trial) {
    double ua, ub;
    rng_pair(r, &ua, &ub);
    double a = 2.0 * ua - 1.0, b = 2.0 * ub - 1.0;
    double s = a * a + b * b;
    if (!(s > 0.0 && s <= 1.0)) continue;
    *cph = (a * a - b * b) / s;
    *sph = 2.0 * a * b / s;
    return trial;
  }
  *cph = 1.0; *sph = 0.0;
  return 0;
}

/* New direction at polar angle theta (cos ct) and azimuth phi about the old direction u. */
static void rotate_about(double *u, double ct, double cph, double sph) {
  double st = sqrt(fmax(0.0, (1.0 - ct) * (1.0 + ct)));
  double dx = st * cph, dy = st * sph, dz = ct;
  double ux = u[0], uy = u[1], uz = u[2];
  double perp2 = ux * ux + uy * uy;
  if (perp2 > 0.0) {
    double perp = sqrt(perp2);
    u[0] = (ux * uz * dx - uy * dy) / perp + ux * dz;
    u[1] = (uy * uz * dx + ux * dy) / perp + uy * dz;
    u[2] = -perp * dx + uz * dz;
  } else if (uz >= 0.0) {
    u[0] = dx; u[1] = dy; u[2] = dz;
  } else {
    u[0] = dx; u[1] = -dy; u[2] = -dz;
  }
}

int o_kahn_sample(double E, uint64_t seed, int64_t tid0, int64_t n, double *eta, double *cost) {
  for (int64_t i = 0; i < n; ++i) {
    ORng r = {seed, tid0 + i, 1u, 0u};
    if (!kahn(E, &r, &eta[i], &cost[i])) return -1;
  }
  return 0;
}

/* ------------------------------------------------------------------ source */

/* Source record (16 doubles): pos[3], spot sigma, has_z, z0, z1, isotropic, dir[3],
 * energy kind (0 mono, 1 uniform, 2 log-uniform), e0, e1, (unused). */
static void gen_source(const double *src, uint64_t seed, int64_t tid, double *pos, double *dir, double *E) {
  ORng r = {seed, tid, 0u, 0u};
  pos[0] = src[0]; pos[1] = src[1]; pos[2] = src[2];
  if (src[3] > 0.0) {
    /* Marsaglia polar method (one block per trial) */
    for (int trial = 0; trial < 1000; ++trial) {
      double ua, ub;
      rng_pair(&r, &ua, &ub);
      double a = 2.0 * ua - 1.0, b = 2.0 * ub - 1.0;
      double s = a * a + b * b;
      if (!(s > 0.0 && s < 1.0)) continue;
      double f = sqrt(-2.0 * log(s) / s);
      pos[0] += src[3] * (a * f);
      pos[1] += src[3] * (b * f);
      break;
    }
  }
  if (src[4] != 0.0) pos[2] = src[5] + (src[6] - src[5]) * rng_u(&r);
  if (src[7] != 0.0) {
    double ct = 2.0 * rng_u(&r) - 1.0;
    double cph, sph;
    azimuth(&r, &cph, &sph);
    double st = sqrt(fmax(0.0, (1.0 - ct) * (1.0 + ct)));
    dir[0] = st * cph; dir[1] = st * sph; dir[2] = ct;
  } else {
    dir[0] = src[8]; dir[1] = src[9]; dir[2] = src[10];
  }
  int ek = (int)src[11];
  if (ek == 0) *E = src[12];
  else if (ek == 1) *E = src[12] + (src[13] - src[12]) * rng_u(&r);
  else *E = src[12] * exp(rng_u(&r) * log(src[13] / src[12]));
}

void o_source_sample(const double *src, uint64_t seed, int64_t tid0, int64_t n, double *pos, double *dir, double *E) {
  for (int64_t i = 0; i < n; ++i) gen_source(src, seed, tid0 + i, pos + 3 * i, dir + 3 * i, E + i);
}

/* ------------------------------------------------------------------ transport */

/* Optional record of one history (o_transport_trace): for each step the state before it
 * (position, direction, energy, path, free path Y / mu) and its outcome (step length,
 * limiter, event), and every (leaf, limiter, event) record in the order it is hashed.
 * Recording stops at the capacities; the history itself runs to its end. */
typedef struct {
  int64_t cap, n, caprec, nrec;
  double *pos, *dir, *E, *step, *sphys;
  int *path, *depth, *lim, *ev;
  int32_t *rec;
} OTrace;

static void trace_state(OTrace *tr, const double *x, const double *u, double E, const int *path, int depth,
                        double sphys) {
  if (!tr || tr->n >= tr->cap) return;
  int64_t n = tr->n;
  memcpy(tr->pos + 3 * n, x, 3 * sizeof(double));
  memcpy(tr->dir + 3 * n, u, 3 * sizeof(double));
  tr->E[n] = E;
  memcpy(tr->path + O_DMAX * n, path, O_DMAX * sizeof(int));
  tr->depth[n] = depth;
  tr->sphys[n] = sphys;
}

static void trace_outcome(OTrace *tr, double s, int lim, int ev) {
  if (!tr || tr->n >= tr->cap) return;
  tr->step[tr->n] = s;
  tr->lim[tr->n] = lim;
  tr->ev[tr->n] = ev;
  tr->n++;
}

/* hash_step, with the record kept in the trace */
static uint64_t record(OTrace *tr, uint64_t h, int32_t leaf, int32_t limiter, int32_t event) {
  if (tr && tr->nrec < tr->caprec) {
    tr->rec[3 * tr->nrec] = leaf;
    tr->rec[3 * tr->nrec + 1] = limiter;
    tr->rec[3 * tr->nrec + 2] = event;
    tr->nrec++;
  }
  return hash_step(h, leaf, limiter, event);
}

/* One history (Algorithm 1 extended with the gamma interactions).  Deposits
 * go to tally[nv] rows per batch: columns 0..nv-1 per volume, nv = escaped
 * energy, nv+1 = source energy.  tr (may be NULL) records the history. */
static void transport_one(const OGeom *g, const double *src, uint64_t seed, int64_t tid, double cutoff, int64_t max_steps,
                          double *tally_row, uint64_t *cnt, uint64_t *hash_out, double *len_out, OTrace *tr) {
  const int nv = g->nvol;
  double x[3], u[3], E;
  gen_source(src, seed, tid, x, u, &E);
  tally_row[nv + 1] += E;
  cnt[C_TRACKS]++;
  uint64_t h = FNV_OFFSET;
  double len = 0.0;
  int path[O_DMAX];
  for (int k = 0; k < O_DMAX; ++k) path[k] = -1;
  int depth = locate_impl(g, x, u, path, cnt);
  if (depth == 0) {
    cnt[C_ESCAPED]++;
    tally_row[nv] += E;
    h = record(tr, h, -1, LIM_MOTHER, EV_ESCAPE);
    if (hash_out) *hash_out = h;
    if (len_out) *len_out = 0.0;
    return;
  }
  ORng rp = {seed, tid, 1u, 0u};
  double Y = -log(rng_u(&rp));
  int nzero = 0;
  int64_t steps = 0;
  for (;;) {
    if (steps >= max_steps) {
      cnt[C_STEPLIMIT]++;
      h = record(tr, h, path[depth - 1], LIM_STEPLIMIT, EV_STEPLIMIT);
      break;
    }
    int leaf = path[depth - 1];
    double mu, mupe;
    mu_lookup(&g->mat[g->vol[leaf].mat], E, &mu, &mupe);
    double sphys = mu > 0.0 ? Y / mu : O_INF;
    trace_state(tr, x, u, E, path, depth, sphys);
    int lim;
    double sgeo = geom_step(g, path, depth, x, u, &lim, NULL, cnt);
    ++steps;
    cnt[C_STEPS]++;
    if (sgeo <= sphys) {
      /* boundary: S_j = S_{j-1} + (t_j - t_{j-1}) mu_j */
      x[0] += sgeo * u[0]; x[1] += sgeo * u[1]; x[2] += sgeo * u[2];
      len += sgeo;
      if (mu > 0.0) { Y = Y - sgeo * mu; if (Y < 0.0) Y = 0.0; }
      cnt[C_GEOM]++;
      depth = relocate_impl(g, path, depth, x, u, cnt);
      if (sgeo <= kHalf) ++nzero; else nzero = 0;
      if (depth > 0 && nzero >= 10) {
        x[0] += 100.0 * kTol * u[0]; x[1] += 100.0 * kTol * u[1]; x[2] += 100.0 * kTol * u[2];
        len += 100.0 * kTol;
        cnt[C_PUSH]++;
        nzero = 0;
        depth = relocate_impl(g, path, depth, x, u, cnt);
        h = record(tr, h, depth > 0 ? path[depth - 1] : -1, LIM_PUSH, EV_PUSH);
      }
      if (depth == 0) {
        cnt[C_ESCAPED]++;
        tally_row[nv] += E;
        h = record(tr, h, -1, lim, EV_ESCAPE);
        trace_outcome(tr, sgeo, lim, EV_ESCAPE);
        break;
      }
      h = record(tr, h, path[depth - 1], lim, EV_NONE);
      trace_outcome(tr, sgeo, lim, EV_NONE);
      continue;
    }
    /* interaction at T = t_{j-1} + (Y - S_{j-1}) / mu_j */
    x[0] += sphys * u[0]; x[1] += sphys * u[1]; x[2] += sphys * u[2];
    len += sphys;
    nzero = 0;
    cnt[C_PHYS]++;
    /* one block per interaction: U chooses the process, W gives the next free path */
    double U, W;
    rng_pair(&rp, &U, &W);
    if (U * mu < mupe) {
      cnt[C_PHOTO]++;
      tally_row[leaf] += E;
      h = record(tr, h, leaf, LIM_PHYS, EV_PHOTO);
      trace_outcome(tr, sphys, LIM_PHYS, EV_PHOTO);
      break;
    }
    cnt[C_COMPTON]++;
    double eta, cost, cph, sph;
    kahn(E, &rp, &eta, &cost);
    azimuth(&rp, &cph, &sph);
    rotate_about(u, cost, cph, sph);
    double E1 = E / eta;
    if (E1 < cutoff) {
      cnt[C_CUTOFF]++;
      tally_row[leaf] += E;
      h = record(tr, h, leaf, LIM_PHYS, EV_CUTOFF);
      trace_outcome(tr, sphys, LIM_PHYS, EV_CUTOFF);
      break;
    }
    tally_row[leaf] += E - E1;
    E = E1;
    Y = -log(W);
    h = record(tr, h, leaf, LIM_PHYS, EV_COMPTON);
    trace_outcome(tr, sphys, LIM_PHYS, EV_COMPTON);
  }
  if (hash_out) *hash_out = h;
  if (len_out) *len_out = len;
}

/* Transport n tracks with ids tid0 .. tid0+n-1.  tally: nb x (nv + 2) doubles,
 * row = track id mod nb.  counters: O_NCOUNT uint64.  hashes / lengths may be NULL.
 * nthreads <= 0 uses the OpenMP default.  Returns the threads used. */
int o_transport(int gi, const double *src, uint64_t seed, int64_t tid0, int64_t n, double cutoff, int64_t max_steps,
                int nb, double *tally, uint64_t *counters, uint64_t *hashes, double *lengths, int nthreads) {
  const OGeom *g = G[gi];
  const int64_t stride = (int64_t)g->nvol + 2;
  int used = 1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
  used = nthreads > 0 ? nthreads : omp_get_max_threads();
#endif
  double **tl = (double **)calloc((size_t)used, sizeof(double *));
  uint64_t **cl = (uint64_t **)calloc((size_t)used, sizeof(uint64_t *));
  for (int t = 0; t < used; ++t) {
    tl[t] = (double *)calloc((size_t)nb * stride, sizeof(double));
    cl[t] = (uint64_t *)calloc(O_NCOUNT, sizeof(uint64_t));
  }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(used)
#endif
  for (int64_t i = 0; i < n; ++i) {
    int t = 0;
#ifdef _OPENMP
    t = omp_get_thread_num();
#endif
    int64_t tid = tid0 + i;
    double *row = tl[t] + (tid % nb) * stride;
    transport_one(g, src, seed, tid, cutoff, max_steps, row, cl[t], hashes ? &hashes[i] : NULL, lengths ? &lengths[i] : NULL,
                  NULL);
  }
  for (int t = 0; t < used; ++t) {
    for (int64_t k = 0; k < (int64_t)nb * stride; ++k) tally[k] += tl[t][k];
    for (int k = 0; k < O_NCOUNT; ++k) counters[k] += cl[t][k];
    free(tl[t]); free(cl[t]);
  }
  free(tl); free(cl);
  return used;
}

/* Algorithm 1 as printed: T = G^{-1}(Y) along the ray from p in direction v at
 * fixed energy E, no interactions.  Returns +inf when the ray leaves the world
 * first.  Also reports the number of boundary steps taken. */
double o_free_path(int gi, const double *p, const double *v, double E, double Y, int64_t *n_steps) {
  const OGeom *g = G[gi];
  int path[O_DMAX];
  double x[3] = {p[0], p[1], p[2]};
  for (int k = 0; k < O_DMAX; ++k) path[k] = -1;
  int depth = locate_impl(g, x, v, path, NULL);
  double t = 0.0, S = 0.0;
  int64_t steps = 0;
  if (Y <= 0.0) { if (n_steps) *n_steps = 0; return 0.0; }
  while (depth > 0 && steps < 100000000) {
    double mu, mupe;
    mu_lookup(&g->mat[g->vol[path[depth - 1]].mat], E, &mu, &mupe);
    int lim;
    double s = geom_step(g, path, depth, x, v, &lim, NULL, NULL);
    ++steps;
    if (mu > 0.0 && S + s * mu >= Y) {
      if (n_steps) *n_steps = steps;
      return t + (Y - S) / mu;
    }
    S += s * mu;
    t += s;
    x[0] = p[0] + t * v[0]; x[1] = p[1] + t * v[1]; x[2] = p[2] + t * v[2];
    depth = relocate_impl(g, path, depth, x, v, NULL);
  }
  if (n_steps) *n_steps = steps;
  return O_INF;
}

/* o_free_path for n rays (pos, dir: n x 3 row-major), OpenMP over rays; returns the threads used. */
int o_free_path_many(int gi, int64_t n, const double *pos, const double *dir, double E, const double *Y, double *T,
                     int64_t *n_steps, int nthreads) {
  int used = 1;
#ifdef _OPENMP
  used = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 64) num_threads(used)
#endif
  for (int64_t i = 0; i < n; ++i) T[i] = o_free_path(gi, pos + 3 * i, dir + 3 * i, E, Y[i], n_steps ? n_steps + i : NULL);
  return used;
}

/* ------------------------------------------------------------------ batch helpers for the tests */

/* pos, dir: n x 3 row-major; depth: n; path: n x O_DMAX row-major. */
void o_locate_many(int gi, int64_t n, const double *pos, const double *dir, int *depth, int *path) {
  for (int64_t i = 0; i < n; ++i) depth[i] = o_locate(gi, pos + 3 * i, dir + 3 * i, path + O_DMAX * i);
}

/* proposed may be NULL (+inf). */
void o_compute_step_many(int gi, int64_t n, const double *pos, const double *dir, const int *depth, const int *path,
                         const double *proposed, double *step, int *limiter, double *safety) {
  for (int64_t i = 0; i < n; ++i) {
    if (depth[i] <= 0) { step[i] = NAN; limiter[i] = -99; safety[i] = NAN; continue; }
    o_compute_step(gi, depth[i], path + O_DMAX * i, pos + 3 * i, dir + 3 * i, proposed ? proposed[i] : O_INF,
                   &step[i], &limiter[i], &safety[i]);
  }
}

/* Per-step trace of one history (debugging aid for parity failures): transport_one itself
 * run with a recorder, so the trace is the history the transport computes.  For every step
 * the state before it (position, direction, energy, path, Y / mu) and its outcome (step
 * length, limiter, event of the step); every hashed (leaf, limiter, event) record in order
 * (records: 3 int32 each, capacity 2 cap + 2); the history's hash, path length and step
 * count.  Returns the steps recorded (at most cap). */
int o_transport_trace(int gi, const double *src, uint64_t seed, int64_t tid, double cutoff, int64_t max_steps,
                      int64_t cap, double *pos, double *dir, double *E_out, int *paths, int *depth_out, double *steps,
                      int *limiters, double *sphys_out, int *events, int32_t *records, int64_t *n_records,
                      uint64_t *hash_out, double *len_out, int64_t *n_steps) {
  const OGeom *g = G[gi];
  OTrace tr = {cap, 0, 2 * cap + 2, 0, pos, dir, E_out, steps, sphys_out, paths, depth_out, limiters, events, records};
  double *row = (double *)calloc((size_t)g->nvol + 2, sizeof(double));
  uint64_t cnt[O_NCOUNT] = {0};
  transport_one(g, src, seed, tid, cutoff, max_steps, row, cnt, hash_out, len_out, &tr);
  free(row);
  *n_records = tr.nrec;
  *n_steps = (int64_t)cnt[C_STEPS];
  return (int)tr.n;
}

/* The direction rotation of a Compton scatter (exported for its pins): u turned to polar
 * cosine ct and azimuth (cph, sph) about itself. */
void o_rotate(const double *u_in, double ct, double cph, double sph, double *u_out) {
  double u[3] = {u_in[0], u_in[1], u_in[2]};
  rotate_about(u, ct, cph, sph);
  memcpy(u_out, u, sizeof(u));
}
