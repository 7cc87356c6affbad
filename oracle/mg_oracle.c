/*
 * mg_oracle.c -- plain, slow FP64 CPU geometric multigrid for the 3-D Poisson
 * equation of self-gravity, written step by step from Tomida & Stone,
 * "The Athena++ AMR Framework: Multigrid Solvers for Self-Gravity" (2023):
 * the discretisation of Sec. 2.1, the red-black SOR smoother of Sec. 2.2,
 * the operators of Sec. 2.3.1, the coarsest-level solver of Sec. 2.3.2,
 * the V-cycle (Algorithm 1), full multigrid (Algorithm 2), the full
 * approximation scheme (Algorithm 3), the boundary rules of Sec. 2.3.6, the
 * stopping rule of Sec. 2.3.7, the multipole boundary of App. A and the
 * cell-centred gravitational acceleration of Sec. 3.2.3.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the correctness oracle for the CUDA
 * library.  It shares no code, header, table or helper with the CUDA path and
 * nothing in the product links it: only the tests, the smoke check and the
 * CPU-baseline leg of bench.py load it.
 *
 * Storage follows the paper's own data structure (Sec. 3.2.1): every level
 * array carries one ghost layer (N_G = 1), so a level of nx*ny*nz active cells
 * is an (nx+2)*(ny+2)*(nz+2) array, x fastest.  Ghost values are (re)filled
 * from the boundary rule before every use, exactly as the paper refreshes
 * ghosts before every colour of the smoother.
 *
 * Readings where the paper is silent (each one is also listed in the design
 * notes of the repository):
 *  - red = (i+j+k) even with 0-based active indices; red is updated first;
 *  - edge and corner ghosts: the face rule is applied along x, then y, then z
 *    (a ghost of a ghost), so 27-point prolongation stencils are defined;
 *  - coarse levels of the correction scheme use the homogeneous counterpart of
 *    the finest-level rule (periodic -> periodic, fixed/open -> zero fixed,
 *    zero gradient -> zero gradient);
 *  - the 1-cell coarsest level is solved exactly with its ghosts eliminated;
 *    when it is singular (periodic, zero gradient) its starting value is kept,
 *    which is 0 for a correction;
 *  - during FMG every level uses the physical boundary rule; for open
 *    boundaries the multipole potential is evaluated at each level's own face
 *    points;
 *  - the stopping test uses ||d||/||f|| with volume-weighted RMS norms.
 *
 * Arithmetic is plain IEEE double; the library is compiled without
 * floating-point contraction so its rounding is the same on every host.
 * Sums run serially in z, y, x order.  Only the per-colour stencil loops are
 * spread over OpenMP threads; every cell of one colour is independent, so the
 * thread count does not change any result.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Status codes (same numbers as the library's public ones, defined here on
 * their own). */
enum {
  ORC_OK = 0,
  ORC_ERR_ARG = 1,
  ORC_ERR_OOM = 2,
  ORC_ERR_NOT_CONVERGED = 4,
  ORC_ERR_DIVERGED = 5
};

/* Boundary kinds, Sec. 2.3.6.  BC_MIXED: a rule of its own on each face
 * (periodic on both faces of an axis, fixed b_face or zero gradient), given to
 * the entry points as a 12-double descriptor in place of the face arrays: the
 * six kinds (x-, x+, y-, y+, z-, z+) followed by the six values b_face (read
 * on fixed faces only). */
enum { BC_PERIODIC = 0, BC_FIXED = 1, BC_ZEROGRAD = 2, BC_OPEN = 3, BC_FACES = 4, BC_MIXED = 5 };

/* Coarse-grid schemes. */
enum { CYCLE_CORRECTION = 0, CYCLE_FAS = 1 };

typedef struct {
  int kind;
  double value;          /* BC_FIXED: the boundary value b on every face    */
  const double *face[6]; /* BC_OPEN / BC_FACES: value on the domain surface */
  int fk[6];             /* BC_MIXED: the kind of each face                 */
  double fv[6];          /* BC_MIXED: b on each fixed face                  */
} Bc;

/* Read a BC_MIXED descriptor into b; a periodic face needs a periodic
 * opposite face, and only periodic, fixed and zero-gradient faces exist. */
static int mixed_from(const double *desc, Bc *b) {
  if (!desc) return 1;
  b->kind = BC_MIXED;
  for (int q = 0; q < 6; ++q) {
    const double k = desc[q];
    if (k != (double)BC_PERIODIC && k != (double)BC_FIXED && k != (double)BC_ZEROGRAD) return 1;
    b->fk[q] = (int)k;
    b->fv[q] = desc[6 + q];
  }
  for (int a = 0; a < 3; ++a)
    if ((b->fk[2 * a] == BC_PERIODIC) != (b->fk[2 * a + 1] == BC_PERIODIC)) return 1;
  return 0;
}

/* Whether a rule fixes the zero point of the potential (Sec. 2.3.6): some
 * face carries a value. */
static int sets_zero_point(const Bc *bc) {
  if (bc->kind != BC_MIXED) return !(bc->kind == BC_PERIODIC || bc->kind == BC_ZEROGRAD);
  for (int q = 0; q < 6; ++q)
    if (bc->fk[q] == BC_FIXED) return 1;
  return 0;
}

typedef struct {
  int nx, ny, nz;
  double h;
  double *u;  /* potential (finest) or correction (coarse), with ghosts */
  double *f;  /* right-hand side, ghosts unused                          */
  double *d;  /* defect scratch                                          */
  double *ur; /* FAS: restricted potential                               */
} Level;

static size_t padded_size(int nx, int ny, int nz) {
  return (size_t)(nx + 2) * (size_t)(ny + 2) * (size_t)(nz + 2);
}

/* Index of padded cell (i, j, k), i, j, k in [0, n+1]; active cells are 1..n. */
static size_t pidx(int nx, int ny, int i, int j, int k) {
  return ((size_t)k * (size_t)(ny + 2) + (size_t)j) * (size_t)(nx + 2) + (size_t)i;
}

/* Index of a point on a face array.  Faces 0/1 are x-lo/x-hi indexed by the
 * padded (j, k); faces 2/3 are y-lo/y-hi indexed by (i, k); faces 4/5 are
 * z-lo/z-hi indexed by (i, j).  Each face array has (n_a+2)*(n_b+2) entries
 * so that the extended points used by edge and corner ghosts exist. */
static size_t fidx(int face, int nx, int ny, int a, int b) {
  if (face < 2) return (size_t)b * (size_t)(ny + 2) + (size_t)a;
  return (size_t)b * (size_t)(nx + 2) + (size_t)a;
}

static double face_value(const Bc *bc, int face, size_t idx) {
  if (bc->kind == BC_FIXED) return bc->value;
  if (bc->kind == BC_MIXED) return bc->fv[face];
  return bc->face[face][idx];
}

/* Sec. 2.3.6: periodic and zero-gradient ghosts are copies of cell centres;
 * fixed and isolated ghosts are set so that the average of the ghost and the
 * adjacent active cell -- the value on the domain surface -- equals the
 * boundary value b, i.e. ghost = 2 b - active. */
static double ghost_of(const Bc *bc, int face, size_t fi, double adjacent, double wrapped) {
  switch (bc->kind == BC_MIXED ? bc->fk[face] : bc->kind) {
    case BC_PERIODIC: return wrapped;
    case BC_ZEROGRAD: return adjacent;
    default: return 2.0 * face_value(bc, face, fi) - adjacent;
  }
}

static void fill_ghosts(const Level *L, double *a, const Bc *bc) {
  const int nx = L->nx, ny = L->ny, nz = L->nz;
  /* x faces over active j, k */
  for (int k = 1; k <= nz; ++k)
    for (int j = 1; j <= ny; ++j) {
      double first = a[pidx(nx, ny, 1, j, k)], last = a[pidx(nx, ny, nx, j, k)];
      a[pidx(nx, ny, 0, j, k)] = ghost_of(bc, 0, fidx(0, nx, ny, j, k), first, last);
      a[pidx(nx, ny, nx + 1, j, k)] = ghost_of(bc, 1, fidx(1, nx, ny, j, k), last, first);
    }
  /* y faces over padded i (so x ghosts take part: edges) and active k */
  for (int k = 1; k <= nz; ++k)
    for (int i = 0; i <= nx + 1; ++i) {
      double first = a[pidx(nx, ny, i, 1, k)], last = a[pidx(nx, ny, i, ny, k)];
      a[pidx(nx, ny, i, 0, k)] = ghost_of(bc, 2, fidx(2, nx, ny, i, k), first, last);
      a[pidx(nx, ny, i, ny + 1, k)] = ghost_of(bc, 3, fidx(3, nx, ny, i, k), last, first);
    }
  /* z faces over padded i, j (edges and corners) */
  for (int j = 0; j <= ny + 1; ++j)
    for (int i = 0; i <= nx + 1; ++i) {
      double first = a[pidx(nx, ny, i, j, 1)], last = a[pidx(nx, ny, i, j, nz)];
      a[pidx(nx, ny, i, j, 0)] = ghost_of(bc, 4, fidx(4, nx, ny, i, j), first, last);
      a[pidx(nx, ny, i, j, nz + 1)] = ghost_of(bc, 5, fidx(5, nx, ny, i, j), last, first);
    }
}

/* The homogeneous counterpart of a boundary rule, used for corrections. */
static Bc homogeneous(const Bc *bc) {
  Bc z;
  memset(&z, 0, sizeof z);
  if (bc->kind == BC_MIXED) {
    z.kind = BC_MIXED;
    for (int q = 0; q < 6; ++q) z.fk[q] = bc->fk[q]; /* fixed faces get b = 0 */
  } else if (bc->kind == BC_PERIODIC || bc->kind == BC_ZEROGRAD) {
    z.kind = bc->kind;
  } else {
    z.kind = BC_FIXED;
    z.value = 0.0;
  }
  return z;
}

/* The rule of the coarse correction levels.  By default the homogeneous
 * counterpart above; with `literal` set, Sec. 2.3.6 read word for word: zero
 * fixed values on every coarse level unless the grid is periodic, so a
 * zero-gradient grid's corrections get zero fixed values too. */
static Bc correction_rule(const Bc *bc, int literal) {
  Bc z = homogeneous(bc);
  if (literal && z.kind == BC_ZEROGRAD) {
    z.kind = BC_FIXED;
    z.value = 0.0;
  }
  if (literal && z.kind == BC_MIXED)
    for (int q = 0; q < 6; ++q)
      if (z.fk[q] == BC_ZEROGRAD) z.fk[q] = BC_FIXED;
  return z;
}

/* ---------------------------------------------------------------------- */
/* Smoother: red-black SOR, Eqs. (rbsor1)-(rbsor2), with omega (Sec. 2.3.2). */

static void sor_colour(Level *L, const Bc *bc, double omega, int colour) {
  const int nx = L->nx, ny = L->ny, nz = L->nz;
  const double h2 = L->h * L->h;
  double *u = L->u;
  const double *f = L->f;
  fill_ghosts(L, u, bc);
#pragma omp parallel for schedule(static)
  for (int k = 1; k <= nz; ++k)
    for (int j = 1; j <= ny; ++j)
      for (int i = 1; i <= nx; ++i) {
        if (((i - 1) + (j - 1) + (k - 1)) % 2 != colour) continue;
        size_t c = pidx(nx, ny, i, j, k);
        double s = u[pidx(nx, ny, i - 1, j, k)] + u[pidx(nx, ny, i + 1, j, k)] +
                   u[pidx(nx, ny, i, j - 1, k)] + u[pidx(nx, ny, i, j + 1, k)] +
                   u[pidx(nx, ny, i, j, k - 1)] + u[pidx(nx, ny, i, j, k + 1)];
        u[c] = u[c] + omega * ((s - 6.0 * u[c]) / 6.0 - f[c] * h2 / 6.0);
      }
}

static void smooth(Level *L, const Bc *bc, double omega) {
  sor_colour(L, bc, omega, 0); /* red   */
  sor_colour(L, bc, omega, 1); /* black */
}

/* Defect d = f - L_h u, Eq. (defect) with the 7-point Laplacian of
 * Eq. (discretized2). */
static void defect(Level *L, const Bc *bc, double *d) {
  const int nx = L->nx, ny = L->ny, nz = L->nz;
  const double h2 = L->h * L->h;
  double *u = L->u;
  fill_ghosts(L, u, bc);
#pragma omp parallel for schedule(static)
  for (int k = 1; k <= nz; ++k)
    for (int j = 1; j <= ny; ++j)
      for (int i = 1; i <= nx; ++i) {
        size_t c = pidx(nx, ny, i, j, k);
        double s = u[pidx(nx, ny, i - 1, j, k)] + u[pidx(nx, ny, i + 1, j, k)] +
                   u[pidx(nx, ny, i, j - 1, k)] + u[pidx(nx, ny, i, j + 1, k)] +
                   u[pidx(nx, ny, i, j, k - 1)] + u[pidx(nx, ny, i, j, k + 1)];
        d[c] = L->f[c] - (s - 6.0 * u[c]) / h2;
      }
}

/* L_h u (no source), used by FAS to build the coarse right-hand side. */
static void apply_laplacian(Level *L, double *u, const Bc *bc, double *out) {
  const int nx = L->nx, ny = L->ny, nz = L->nz;
  const double h2 = L->h * L->h;
  fill_ghosts(L, u, bc);
  for (int k = 1; k <= nz; ++k)
    for (int j = 1; j <= ny; ++j)
      for (int i = 1; i <= nx; ++i) {
        double s = u[pidx(nx, ny, i - 1, j, k)] + u[pidx(nx, ny, i + 1, j, k)] +
                   u[pidx(nx, ny, i, j - 1, k)] + u[pidx(nx, ny, i, j + 1, k)] +
                   u[pidx(nx, ny, i, j, k - 1)] + u[pidx(nx, ny, i, j, k + 1)];
        out[pidx(nx, ny, i, j, k)] = (s - 6.0 * u[pidx(nx, ny, i, j, k)]) / h2;
      }
}

/* Restriction I_l^{l-1}, Eq. (restriction): volume-weighted average of the
 * 2x2x2 children; on a uniform grid every weight is the same. */
static void restrict_avg(const Level *F, const double *uf, const Level *C, double *uc) {
  for (int K = 1; K <= C->nz; ++K)
    for (int J = 1; J <= C->ny; ++J)
      for (int I = 1; I <= C->nx; ++I) {
        double sum = 0.0, vol = 0.0;
        for (int c = 0; c < 2; ++c)
          for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
              int i = 2 * (I - 1) + a + 1, j = 2 * (J - 1) + b + 1, k = 2 * (K - 1) + c + 1;
              double dv = 1.0; /* uniform cell volume */
              sum += uf[pidx(F->nx, F->ny, i, j, k)] * dv;
              vol += dv;
            }
        uc[pidx(C->nx, C->ny, I, J, K)] = sum / vol;
      }
}

/* One-dimensional weights of the prolongations, Eq. (trilinear) and the FMG
 * operator I' that follows it: w[n+1] for n = -1, 0, +1, by fine-index parity
 * (even = fine cell on the lower side of its parent). */
static void prolong_weights(int high_order, int odd, double w[3]) {
  if (!high_order) {
    if (!odd) { w[0] = 0.25; w[1] = 0.75; w[2] = 0.0; }
    else      { w[0] = 0.0;  w[1] = 0.75; w[2] = 0.25; }
  } else {
    if (!odd) { w[0] = 5.0 / 32.0;  w[1] = 30.0 / 32.0; w[2] = -3.0 / 32.0; }
    else      { w[0] = -3.0 / 32.0; w[1] = 30.0 / 32.0; w[2] = 5.0 / 32.0; }
  }
}

/* u_f (+)= sum_{a,b,c} w_a w_b w_c u_c(I+a, J+b, K+c).  The coarse ghosts must
 * have been filled by the caller. */
static void prolong(const Level *C, const double *uc, const Level *F, double *uf,
                    int high_order, int add) {
  const int nx = F->nx, ny = F->ny, nz = F->nz;
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double wx[3], wy[3], wz[3];
        prolong_weights(high_order, i % 2, wx);
        prolong_weights(high_order, j % 2, wy);
        prolong_weights(high_order, k % 2, wz);
        int I = i / 2 + 1, J = j / 2 + 1, K = k / 2 + 1; /* padded coarse parent */
        double v = 0.0;
        for (int c = -1; c <= 1; ++c)
          for (int b = -1; b <= 1; ++b)
            for (int a = -1; a <= 1; ++a)
              v += wx[a + 1] * wy[b + 1] * wz[c + 1] *
                   uc[pidx(C->nx, C->ny, I + a, J + b, K + c)];
        size_t o = pidx(nx, ny, i + 1, j + 1, k + 1);
        uf[o] = add ? uf[o] + v : v;
      }
}

/* COARSEST(u, L, f), Sec. 2.3.2; u holds the starting value on entry. */
static void coarsest(Level *L, const Bc *bc) {
  const int nx = L->nx, ny = L->ny, nz = L->nz;
  const double h2 = L->h * L->h;
  if (nx * ny * nz == 1) {
    size_t c = pidx(1, 1, 1, 1, 1);
    if (bc->kind == BC_MIXED) {
      /* A periodic or zero-gradient ghost is u itself, a fixed one 2 b - u:
       * with a fixed faces, sum(ghosts) - 6u = 2 sum(b) - 2 a u = h^2 f.
       * Without a fixed face it is singular, as below. */
      int a = 0;
      double sb = 0.0;
      for (int q = 0; q < 6; ++q)
        if (bc->fk[q] == BC_FIXED) { ++a; sb += bc->fv[q]; }
      if (a > 0) L->u[c] = (2.0 * sb - h2 * L->f[c]) / (2.0 * a);
    } else if (bc->kind == BC_PERIODIC || bc->kind == BC_ZEROGRAD) {
      /* Every ghost equals u itself: the 1-cell system is singular (its
       * right-hand side is 0 once the mean is removed) and any value solves
       * it; the starting value is kept, which is 0 for a correction. */
    } else {
      /* Each of the six ghosts is 2 b_face - u, so the discrete equation
       * sum(2 b_face - u) - 6u = h^2 f gives u = (2 sum b_face - h^2 f)/12. */
      double sb = face_value(bc, 0, fidx(0, 1, 1, 1, 1)) + face_value(bc, 1, fidx(1, 1, 1, 1, 1)) +
                  face_value(bc, 2, fidx(2, 1, 1, 1, 1)) + face_value(bc, 3, fidx(3, 1, 1, 1, 1)) +
                  face_value(bc, 4, fidx(4, 1, 1, 1, 1)) + face_value(bc, 5, fidx(5, 1, 1, 1, 1));
      L->u[c] = (2.0 * sb - h2 * L->f[c]) / 12.0;
    }
    return;
  }
  /* More than one cell: N_0,max red-black Gauss-Seidel sweeps (omega = 1). */
  int nmax = nx > ny ? nx : ny;
  if (nz > nmax) nmax = nz;
  for (int s = 0; s < nmax; ++s) smooth(L, bc, 1.0);
}

/* ---------------------------------------------------------------------- */

typedef struct {
  double omega;
  int pre, post;
  int cycle; /* CYCLE_CORRECTION or CYCLE_FAS */
} CycleOpts;

static void zero_active(Level *L, double *a) {
  memset(a, 0, padded_size(L->nx, L->ny, L->nz) * sizeof(double));
}

/* Algorithm 1 (correction scheme) and Algorithm 3 (FAS) on level l.  bc[l] is
 * the rule for level l; in the correction scheme levels below the top of the
 * cycle use the homogeneous rule hom. */
static void multigrid(Level *lev, int l, const Bc *bcs, const Bc *bc_top, const Bc *hom,
                      const CycleOpts *o) {
  Level *F = &lev[l], *C = &lev[l - 1];
  const Bc *bc_coarse = (o->cycle == CYCLE_FAS) ? &bcs[l - 1] : hom;
  for (int s = 0; s < o->pre; ++s) smooth(F, bc_top, o->omega); /* 1 */
  defect(F, bc_top, F->d);                                      /* 2 */
  restrict_avg(F, F->d, C, C->f);                               /* 3 */
  if (o->cycle == CYCLE_FAS) {
    restrict_avg(F, F->u, C, C->ur);                            /* 4 */
    apply_laplacian(C, C->ur, bc_coarse, C->d);                 /* 5 */
    for (size_t q = 0; q < padded_size(C->nx, C->ny, C->nz); ++q) C->f[q] += C->d[q];
    memcpy(C->u, C->ur, padded_size(C->nx, C->ny, C->nz) * sizeof(double));
  } else {
    zero_active(C, C->u); /* the coarse correction starts from 0 */
  }
  if (l - 1 == 0) coarsest(C, bc_coarse);                       /* 4.1 / 6.1 */
  else multigrid(lev, l - 1, bcs, bc_coarse, hom, o);           /* 4.2 / 6.2 */
  if (o->cycle == CYCLE_FAS) {                                  /* 7 */
    for (size_t q = 0; q < padded_size(C->nx, C->ny, C->nz); ++q) C->u[q] -= C->ur[q];
    fill_ghosts(C, C->u, hom);
  } else {
    fill_ghosts(C, C->u, hom);
  }
  prolong(C, C->u, F, F->u, 0, 1);                              /* 5-6 / 8-9 */
  for (int s = 0; s < o->post; ++s) smooth(F, bc_top, o->omega); /* 7 / 10 */
}

/* Algorithm 2, full multigrid. */
static void fmg(Level *lev, int nlev, const Bc *bcs, const Bc *hom, const CycleOpts *o) {
  for (int l = nlev - 1; l >= 1; --l) restrict_avg(&lev[l], lev[l].f, &lev[l - 1], lev[l - 1].f); /* 1 */
  zero_active(&lev[0], lev[0].u);
  coarsest(&lev[0], &bcs[0]);                                                                  /* 2 */
  for (int l = 1; l < nlev; ++l) {
    fill_ghosts(&lev[l - 1], lev[l - 1].u, &bcs[l - 1]);
    prolong(&lev[l - 1], lev[l - 1].u, &lev[l], lev[l].u, 1, 0);                             /* 3 */
    multigrid(lev, l, bcs, &bcs[l], hom, o);                                                 /* 4 */
  }
}

/* Volume-weighted RMS over the active cells, Eq. (threshold). */
static double rms(const Level *L, const double *a) {
  double s = 0.0;
  for (int k = 1; k <= L->nz; ++k)
    for (int j = 1; j <= L->ny; ++j)
      for (int i = 1; i <= L->nx; ++i) {
        double v = a[pidx(L->nx, L->ny, i, j, k)];
        s += v * v;
      }
  return sqrt(s / ((double)L->nx * L->ny * L->nz));
}

static double mean_active(const Level *L, const double *a) {
  double s = 0.0;
  for (int k = 1; k <= L->nz; ++k)
    for (int j = 1; j <= L->ny; ++j)
      for (int i = 1; i <= L->nx; ++i) s += a[pidx(L->nx, L->ny, i, j, k)];
  return s / ((double)L->nx * L->ny * L->nz);
}

/* ---------------------------------------------------------------------- */
/* App. A: multipole expansion. */

/* Real spherical harmonic Y_lm at the unit vector (x, y, z), from the
 * Cartesian table of App. A. */
double orc_ylm(int l, int m, double x, double y, double z) {
  const double pi = 3.14159265358979323846;
  switch (l) {
    case 0: return sqrt(1.0 / (4.0 * pi));
    case 1:
      switch (m) {
        case -1: return sqrt(3.0 / (4.0 * pi)) * y;
        case 0: return sqrt(3.0 / (4.0 * pi)) * z;
        case 1: return sqrt(3.0 / (4.0 * pi)) * x;
      }
      break;
    case 2:
      switch (m) {
        case -2: return sqrt(15.0 / (4.0 * pi)) * x * y;
        case -1: return sqrt(15.0 / (4.0 * pi)) * y * z;
        case 0: return sqrt(5.0 / (16.0 * pi)) * (3.0 * z * z - 1.0);
        case 1: return sqrt(15.0 / (4.0 * pi)) * x * z;
        case 2: return sqrt(15.0 / (4.0 * pi)) * (x * x - y * y) / 2.0;
      }
      break;
    case 3:
      switch (m) {
        case -3: return sqrt(35.0 / (32.0 * pi)) * y * (3.0 * x * x - y * y);
        case -2: return sqrt(105.0 / (4.0 * pi)) * x * y * z;
        case -1: return sqrt(21.0 / (32.0 * pi)) * y * (5.0 * z * z - 1.0);
        case 0: return sqrt(7.0 / (16.0 * pi)) * z * (5.0 * z * z - 3.0);
        case 1: return sqrt(21.0 / (32.0 * pi)) * x * (5.0 * z * z - 1.0);
        case 2: return sqrt(105.0 / (4.0 * pi)) * z * (x * x - y * y) / 2.0;
        case 3: return sqrt(35.0 / (32.0 * pi)) * x * (x * x - 3.0 * y * y);
      }
      break;
    case 4:
      switch (m) {
        case -4: return sqrt(315.0 / (4.0 * pi)) * x * y * (x * x - y * y) / 2.0;
        case -3: return sqrt(315.0 / (32.0 * pi)) * y * z * (3.0 * x * x - y * y);
        case -2: return sqrt(45.0 / (16.0 * pi)) * x * y * (7.0 * z * z - 1.0);
        case -1: return sqrt(45.0 / (32.0 * pi)) * y * z * (7.0 * z * z - 3.0);
        case 0: return sqrt(9.0 / (256.0 * pi)) * (35.0 * z * z * z * z - 30.0 * z * z + 3.0);
        case 1: return sqrt(45.0 / (32.0 * pi)) * x * z * (7.0 * z * z - 3.0);
        case 2: return sqrt(45.0 / (16.0 * pi)) * (x * x - y * y) * (7.0 * z * z - 1.0) / 2.0;
        case 3: return sqrt(315.0 / (32.0 * pi)) * x * z * (x * x - 3.0 * y * y);
        case 4:
          return sqrt(315.0 / (4.0 * pi)) *
                 (x * x * (x * x - 3.0 * y * y) - y * y * (3.0 * x * x - y * y)) / 8.0;
      }
      break;
  }
  return 0.0;
}

/* Cell-centre coordinate of active index i on an axis of n cells: the domain
 * is centred on the origin, so x_i = (i + 1/2 - n/2) h. */
static double centre(int i, int n, double h) { return ((double)i + 0.5 - 0.5 * (double)n) * h; }

/* Multipole moments Q_lm (App. A) of rho on an nx*ny*nz grid of spacing h,
 * about `origin` or, if use_com, about the centre of mass (written back to
 * origin).  Q has (lmax+1)^2 entries ordered l*l + (m + l).  A grid with zero
 * total mass keeps the given origin. */
void orc_multipole_moments(int nx, int ny, int nz, double h, const double *rho, int lmax,
                           int use_com, double origin[3], double *Q) {
  const double pi = 3.14159265358979323846;
  const double dv = h * h * h;
  if (use_com) {
    double m = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          double r = rho[((size_t)k * ny + j) * nx + i];
          m += r * dv;
          mx += r * dv * centre(i, nx, h);
          my += r * dv * centre(j, ny, h);
          mz += r * dv * centre(k, nz, h);
        }
    if (m != 0.0) {
      origin[0] = mx / m;
      origin[1] = my / m;
      origin[2] = mz / m;
    }
  }
  for (int q = 0; q < (lmax + 1) * (lmax + 1); ++q) Q[q] = 0.0;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double r0 = rho[((size_t)k * ny + j) * nx + i];
        double x = centre(i, nx, h) - origin[0];
        double y = centre(j, ny, h) - origin[1];
        double z = centre(k, nz, h) - origin[2];
        double r = sqrt(x * x + y * y + z * z);
        for (int l = 0; l <= lmax; ++l) {
          double rl = 1.0;
          for (int p = 0; p < l; ++p) rl *= r;
          for (int m = -l; m <= l; ++m) {
            double y_lm = (r > 0.0) ? orc_ylm(l, m, x / r, y / r, z / r)
                                    : (l == 0 ? orc_ylm(0, 0, 0, 0, 0) : 0.0);
            Q[l * l + m + l] += r0 * dv * sqrt(4.0 * pi / (2.0 * l + 1.0)) * rl * y_lm;
          }
        }
      }
}

/* Exterior potential of App. A at (x, y, z) about `origin`.  The sign is that
 * of the Poisson equation with f = 4 pi G rho (attractive gravity): the l = 0
 * term is -G M / r. */
double orc_multipole_potential(const double *Q, int lmax, double G, const double origin[3],
                               double x, double y, double z) {
  const double pi = 3.14159265358979323846;
  x -= origin[0];
  y -= origin[1];
  z -= origin[2];
  double r = sqrt(x * x + y * y + z * z);
  double phi = 0.0;
  for (int l = 0; l <= lmax; ++l) {
    double rl1 = r;
    for (int p = 0; p < l; ++p) rl1 *= r;
    for (int m = -l; m <= l; ++m)
      phi += Q[l * l + m + l] / rl1 * sqrt(4.0 * pi / (2.0 * l + 1.0)) * orc_ylm(l, m, x / r, y / r, z / r);
  }
  return -G * phi;
}

/* Boundary values of the six faces of a level (nx, ny, nz, h) for an open
 * boundary: the multipole potential at every padded face point.  faces holds
 * 2*(ny+2)(nz+2) + 2*(nx+2)(nz+2) + 2*(nx+2)(ny+2) values, faces 0..5 in turn. */
void orc_open_faces(int nx, int ny, int nz, double h, const double *Q, int lmax, double G,
                    const double origin[3], double *faces) {
  double X = 0.5 * nx * h, Y = 0.5 * ny * h, Z = 0.5 * nz * h;
  size_t off = 0;
  for (int face = 0; face < 6; ++face) {
    int na, nb;
    if (face < 2) { na = ny; nb = nz; }
    else if (face < 4) { na = nx; nb = nz; }
    else { na = nx; nb = ny; }
    for (int b = 0; b <= nb + 1; ++b)
      for (int a = 0; a <= na + 1; ++a) {
        double x, y, z;
        double pa = ((double)a - 0.5 - 0.5 * na) * h, pb = ((double)b - 0.5 - 0.5 * nb) * h;
        double side = (face % 2 == 0) ? -1.0 : 1.0;
        if (face < 2) { x = side * X; y = pa; z = pb; }
        else if (face < 4) { x = pa; y = side * Y; z = pb; }
        else { x = pa; y = pb; z = side * Z; }
        faces[off + (size_t)b * (na + 2) + a] = orc_multipole_potential(Q, lmax, G, origin, x, y, z);
      }
    off += (size_t)(na + 2) * (nb + 2);
  }
}

static size_t faces_total(int nx, int ny, int nz) {
  return 2 * (size_t)(ny + 2) * (nz + 2) + 2 * (size_t)(nx + 2) * (nz + 2) +
         2 * (size_t)(nx + 2) * (ny + 2);
}

static void faces_split(int nx, int ny, int nz, const double *faces, const double *out[6]) {
  size_t off = 0;
  for (int face = 0; face < 6; ++face) {
    out[face] = faces + off;
    if (face < 2) off += (size_t)(ny + 2) * (nz + 2);
    else if (face < 4) off += (size_t)(nx + 2) * (nz + 2);
    else off += (size_t)(nx + 2) * (ny + 2);
  }
}

/* ---------------------------------------------------------------------- */
/* Level hierarchy. */

static int is_pow2(int n) { return n >= 1 && (n & (n - 1)) == 0; }

typedef struct {
  int nlev;
  Level *lev;
  Bc *bcs;      /* physical rule per level */
  double **faces; /* per-level face storage (open) */
} Hier;

static void hier_free(Hier *H) {
  if (!H->lev) return;
  for (int l = 0; l < H->nlev; ++l) {
    free(H->lev[l].u);
    free(H->lev[l].f);
    free(H->lev[l].d);
    free(H->lev[l].ur);
    if (H->faces) free(H->faces[l]);
  }
  free(H->lev);
  free(H->bcs);
  free(H->faces);
  memset(H, 0, sizeof *H);
}

static int hier_build(Hier *H, int nx, int ny, int nz, double h) {
  memset(H, 0, sizeof *H);
  int nlev = 1, ax = nx, ay = ny, az = nz;
  while (ax % 2 == 0 && ay % 2 == 0 && az % 2 == 0) {
    ax /= 2; ay /= 2; az /= 2; ++nlev;
  }
  H->nlev = nlev;
  H->lev = calloc((size_t)nlev, sizeof(Level));
  H->bcs = calloc((size_t)nlev, sizeof(Bc));
  H->faces = calloc((size_t)nlev, sizeof(double *));
  if (!H->lev || !H->bcs || !H->faces) return ORC_ERR_OOM;
  for (int l = nlev - 1, s = 0; l >= 0; --l, ++s) {
    Level *L = &H->lev[l];
    L->nx = nx >> s; L->ny = ny >> s; L->nz = nz >> s;
    L->h = h * (double)(1 << s);
    size_t n = padded_size(L->nx, L->ny, L->nz);
    L->u = calloc(n, sizeof(double));
    L->f = calloc(n, sizeof(double));
    L->d = calloc(n, sizeof(double));
    L->ur = calloc(n, sizeof(double));
    if (!L->u || !L->f || !L->d || !L->ur) return ORC_ERR_OOM;
  }
  return ORC_OK;
}

/* Fill the physical rule of every level. */
static int hier_set_bc(Hier *H, int kind, double value, const double *Q, int lmax, double G,
                       const double origin[3], const double *finest_faces) {
  for (int l = 0; l < H->nlev; ++l) {
    Level *L = &H->lev[l];
    Bc *b = &H->bcs[l];
    memset(b, 0, sizeof *b);
    b->kind = kind;
    b->value = value;
    if (kind == BC_MIXED) {
      /* the same face kinds and values on every level (FMG) */
      if (mixed_from(finest_faces, b)) return ORC_ERR_ARG;
    } else if (kind == BC_OPEN || kind == BC_FACES) {
      H->faces[l] = calloc(faces_total(L->nx, L->ny, L->nz), sizeof(double));
      if (!H->faces[l]) return ORC_ERR_OOM;
      if (kind == BC_OPEN) {
        orc_open_faces(L->nx, L->ny, L->nz, L->h, Q, lmax, G, origin, H->faces[l]);
      } else if (l == H->nlev - 1) {
        memcpy(H->faces[l], finest_faces, faces_total(L->nx, L->ny, L->nz) * sizeof(double));
      } else {
        /* Given faces are only defined on the finest level: below it the rule
         * is applied to corrections only, so FMG is not offered here. */
      }
      faces_split(L->nx, L->ny, L->nz, H->faces[l], b->face);
    }
  }
  return ORC_OK;
}

/* The hierarchy of a solve with its physical rule on every level: for open
 * boundaries the moments of rho (App. A) and each level's face values. */
static int hier_with_rules(Hier *H, int nx, int ny, int nz, double h, int bc_kind,
                           double bc_value, const double *given_faces, int lmax, int use_com,
                           const double *origin_in, double four_pi_G, const double *rho,
                           double *origin_out, double *Q_out) {
  int st = hier_build(H, nx, ny, nz, h);
  if (st != ORC_OK) return st;
  const double pi = 3.14159265358979323846;
  double origin[3] = {0.0, 0.0, 0.0};
  double Q[25];
  memset(Q, 0, sizeof Q);
  if (origin_in) memcpy(origin, origin_in, sizeof origin);
  if (bc_kind == BC_OPEN) orc_multipole_moments(nx, ny, nz, h, rho, lmax, use_com, origin, Q);
  if (origin_out) memcpy(origin_out, origin, sizeof origin);
  if (Q_out) memcpy(Q_out, Q, sizeof Q);
  return hier_set_bc(H, bc_kind, bc_value, Q, lmax, four_pi_G / (4.0 * pi), origin, given_faces);
}

/* The face values an open-boundary solve of rho gives level `level` (0 the
 * coarsest) of its hierarchy, exactly as orc_solve sets them up for the FMG
 * ladder (Sec. 2.3.6: each level's own face points).  faces receives
 * faces_total of that level. */
int orc_open_level_faces(int nx, int ny, int nz, double h, const double *rho, int lmax,
                         int use_com, const double *origin_in, double four_pi_G, int level,
                         double *faces) {
  if (!is_pow2(nx) || !is_pow2(ny) || !is_pow2(nz) || h <= 0.0) return ORC_ERR_ARG;
  Hier H;
  int st = hier_with_rules(&H, nx, ny, nz, h, BC_OPEN, 0.0, NULL, lmax, use_com, origin_in,
                           four_pi_G, rho, NULL, NULL);
  if (st == ORC_OK && (level < 0 || level >= H.nlev)) st = ORC_ERR_ARG;
  if (st == ORC_OK) {
    const Level *L = &H.lev[level];
    memcpy(faces, H.faces[level], faces_total(L->nx, L->ny, L->nz) * sizeof(double));
  }
  hier_free(&H);
  return st;
}

/* ---------------------------------------------------------------------- */
/* Whole solve (Sec. 2.3.7): f = 4 pi G rho (mean removed where no boundary
 * fixes the zero point, Sec. 2.3.6), FMG or a given initial guess, then
 * V-cycles on the finest level until ||d||/||f|| < tol, a stall, divergence
 * or max_cycles.  hist[0] is the ratio after FMG (or for the initial guess);
 * hist[n] after the n-th further V-cycle. */
int orc_solve(int nx, int ny, int nz, double h, int bc_kind, double bc_value,
              const double *given_faces, int lmax, int use_com, const double *origin_in,
              double omega, int pre, int post, int mode_fmg, int cycle, int coarse_literal,
              int max_cycles,
              double stall_ratio, double tol, double four_pi_G, const double *rho, double *phi,
              double *hist, int hist_cap, int *n_hist, double *origin_out, double *Q_out) {
  if (!is_pow2(nx) || !is_pow2(ny) || !is_pow2(nz) || h <= 0.0) return ORC_ERR_ARG;
  if (bc_kind < 0 || bc_kind > BC_MIXED || pre < 0 || post < 0 || max_cycles < 0) return ORC_ERR_ARG;
  if (lmax < 0 || lmax > 4 || hist_cap < 1) return ORC_ERR_ARG;
  if (bc_kind == BC_FACES && (mode_fmg || cycle == CYCLE_FAS)) return ORC_ERR_ARG;
  Hier H;
  int st = hier_with_rules(&H, nx, ny, nz, h, bc_kind, bc_value, given_faces, lmax, use_com,
                           origin_in, four_pi_G, rho, origin_out, Q_out);
  if (st != ORC_OK) { hier_free(&H); return st; }
  Level *F = &H.lev[H.nlev - 1];
  Bc hom = correction_rule(&H.bcs[0], coarse_literal);

  /* f = 4 pi G rho */
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i)
        F->f[pidx(nx, ny, i + 1, j + 1, k + 1)] = four_pi_G * rho[((size_t)k * ny + j) * nx + i];
  int mean_free = !sets_zero_point(&H.bcs[0]);
  if (mean_free) {
    double m = mean_active(F, F->f);
    for (int k = 1; k <= nz; ++k)
      for (int j = 1; j <= ny; ++j)
        for (int i = 1; i <= nx; ++i) F->f[pidx(nx, ny, i, j, k)] -= m;
  }
  double fnorm = rms(F, F->f);

  CycleOpts o = {omega, pre, post, cycle};
  if (mode_fmg) {
    fmg(H.lev, H.nlev, H.bcs, &hom, &o);
  } else {
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
          F->u[pidx(nx, ny, i + 1, j + 1, k + 1)] = phi[((size_t)k * ny + j) * nx + i];
  }
  defect(F, &H.bcs[H.nlev - 1], F->d);
  double dn = rms(F, F->d);
  if (fnorm == 0.0) {
    /* No source: measure against the defect of the starting guess instead. */
    fnorm = dn > 0.0 ? dn : 1.0;
  }
  int n = 0;
  hist[n++] = dn / fnorm;
  st = ORC_ERR_NOT_CONVERGED;
  double d0 = hist[0], prev = hist[0];
  int stalls = 0;
  for (int cyc = 0;; ++cyc) {
    double r = hist[n - 1];
    if (isnan(r) || isinf(r) || r > 10.0 * d0) { st = ORC_ERR_DIVERGED; break; }
    if (r < tol) { st = ORC_OK; break; }
    if (stalls >= 2) { st = (tol == 0.0) ? ORC_OK : ORC_ERR_NOT_CONVERGED; break; }
    if (cyc >= max_cycles || n >= hist_cap) { st = ORC_ERR_NOT_CONVERGED; break; }
    multigrid(H.lev, H.nlev - 1, H.bcs, &H.bcs[H.nlev - 1], &hom, &o);
    defect(F, &H.bcs[H.nlev - 1], F->d);
    double rn = rms(F, F->d) / fnorm;
    stalls = (rn > stall_ratio * prev) ? stalls + 1 : 0;
    prev = rn;
    hist[n++] = rn;
  }
  if (mean_free) {
    double m = mean_active(F, F->u);
    for (int k = 1; k <= nz; ++k)
      for (int j = 1; j <= ny; ++j)
        for (int i = 1; i <= nx; ++i) F->u[pidx(nx, ny, i, j, k)] -= m;
  }
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i)
        phi[((size_t)k * ny + j) * nx + i] = F->u[pidx(nx, ny, i + 1, j + 1, k + 1)];
  *n_hist = n;
  hier_free(&H);
  return st;
}

/* ---------------------------------------------------------------------- */
/* Single operators on unpadded (nz, ny, nx) arrays, for per-kernel parity. */

typedef struct {
  Level L;
  Bc bc;
  double *faces;
} OneLevel;

static int one_level(OneLevel *o, int nx, int ny, int nz, double h, int bc_kind, double bc_value,
                     const double *faces) {
  memset(o, 0, sizeof *o);
  o->L.nx = nx; o->L.ny = ny; o->L.nz = nz; o->L.h = h;
  size_t n = padded_size(nx, ny, nz);
  o->L.u = calloc(n, sizeof(double));
  o->L.f = calloc(n, sizeof(double));
  o->L.d = calloc(n, sizeof(double));
  if (!o->L.u || !o->L.f || !o->L.d) return ORC_ERR_OOM;
  o->bc.kind = bc_kind;
  o->bc.value = bc_value;
  if (bc_kind == BC_MIXED) {
    if (mixed_from(faces, &o->bc)) return ORC_ERR_ARG;
  } else if (bc_kind == BC_OPEN || bc_kind == BC_FACES) {
    o->faces = malloc(faces_total(nx, ny, nz) * sizeof(double));
    if (!o->faces) return ORC_ERR_OOM;
    memcpy(o->faces, faces, faces_total(nx, ny, nz) * sizeof(double));
    faces_split(nx, ny, nz, o->faces, o->bc.face);
  }
  return ORC_OK;
}

static void one_free(OneLevel *o) {
  free(o->L.u); free(o->L.f); free(o->L.d); free(o->faces);
}

static void load(const Level *L, double *pad, const double *a) {
  for (int k = 0; k < L->nz; ++k)
    for (int j = 0; j < L->ny; ++j)
      for (int i = 0; i < L->nx; ++i)
        pad[pidx(L->nx, L->ny, i + 1, j + 1, k + 1)] = a[((size_t)k * L->ny + j) * L->nx + i];
}

static void store(const Level *L, const double *pad, double *a) {
  for (int k = 0; k < L->nz; ++k)
    for (int j = 0; j < L->ny; ++j)
      for (int i = 0; i < L->nx; ++i)
        a[((size_t)k * L->ny + j) * L->nx + i] = pad[pidx(L->nx, L->ny, i + 1, j + 1, k + 1)];
}

/* Smoother steps: colours == 0 -> red then black per step; 1 -> red only;
 * 2 -> black only. */
int orc_op_smooth(int nx, int ny, int nz, double h, int bc_kind, double bc_value,
                  const double *faces, double omega, int steps, int colours, double *u,
                  const double *f) {
  OneLevel o;
  int e = one_level(&o, nx, ny, nz, h, bc_kind, bc_value, faces);
  if (e != ORC_OK) { one_free(&o); return e; }
  load(&o.L, o.L.u, u);
  load(&o.L, o.L.f, f);
  for (int s = 0; s < steps; ++s) {
    if (colours == 0) smooth(&o.L, &o.bc, omega);
    else sor_colour(&o.L, &o.bc, omega, colours - 1);
  }
  store(&o.L, o.L.u, u);
  one_free(&o);
  return ORC_OK;
}

int orc_op_defect(int nx, int ny, int nz, double h, int bc_kind, double bc_value,
                  const double *faces, const double *u, const double *f, double *d) {
  OneLevel o;
  int e = one_level(&o, nx, ny, nz, h, bc_kind, bc_value, faces);
  if (e != ORC_OK) { one_free(&o); return e; }
  load(&o.L, o.L.u, u);
  load(&o.L, o.L.f, f);
  defect(&o.L, &o.bc, o.L.d);
  store(&o.L, o.L.d, d);
  one_free(&o);
  return ORC_OK;
}

/* Restriction of an (nz, ny, nx) fine array to (nz/2, ny/2, nx/2). */
int orc_op_restrict(int nx, int ny, int nz, const double *uf, double *uc) {
  OneLevel F, C;
  if (one_level(&F, nx, ny, nz, 1.0, BC_PERIODIC, 0.0, NULL) != ORC_OK ||
      one_level(&C, nx / 2, ny / 2, nz / 2, 2.0, BC_PERIODIC, 0.0, NULL) != ORC_OK) {
    one_free(&F); one_free(&C); return ORC_ERR_OOM;
  }
  load(&F.L, F.L.u, uf);
  restrict_avg(&F.L, F.L.u, &C.L, C.L.u);
  store(&C.L, C.L.u, uc);
  one_free(&F); one_free(&C);
  return ORC_OK;
}

/* Prolongation of a coarse (nz/2, ny/2, nx/2) array to the fine (nz, ny, nx)
 * grid with the coarse ghosts from the given rule.  high_order selects I';
 * add selects u_f += I u_c (correction) over u_f = I u_c. */
int orc_op_prolong(int nx, int ny, int nz, int bc_kind, double bc_value, const double *coarse_faces,
                   int high_order, int add, const double *uc, double *uf) {
  OneLevel F, C;
  int e = one_level(&F, nx, ny, nz, 1.0, BC_PERIODIC, 0.0, NULL);
  if (e == ORC_OK) e = one_level(&C, nx / 2, ny / 2, nz / 2, 2.0, bc_kind, bc_value, coarse_faces);
  if (e != ORC_OK) { one_free(&F); one_free(&C); return e; }
  load(&C.L, C.L.u, uc);
  load(&F.L, F.L.u, uf);
  fill_ghosts(&C.L, C.L.u, &C.bc);
  prolong(&C.L, C.L.u, &F.L, F.L.u, high_order, add);
  store(&F.L, F.L.u, uf);
  one_free(&F); one_free(&C);
  return ORC_OK;
}

/* COARSEST on a single level from a zero guess. */
int orc_op_coarsest(int nx, int ny, int nz, double h, int bc_kind, double bc_value,
                    const double *faces, const double *f, double *u) {
  OneLevel o;
  int e = one_level(&o, nx, ny, nz, h, bc_kind, bc_value, faces);
  if (e != ORC_OK) { one_free(&o); return e; }
  load(&o.L, o.L.f, f);
  coarsest(&o.L, &o.bc);
  store(&o.L, o.L.u, u);
  one_free(&o);
  return ORC_OK;
}

/* One V-cycle of Algorithm 1 (cycle = 0) or Algorithm 3 (cycle = 1) on the
 * finest level of an nx*ny*nz grid, given u and f (f is used as is); `mixed`
 * is the BC_MIXED descriptor (else unused). */
int orc_op_vcycle(int nx, int ny, int nz, double h, int bc_kind, double bc_value,
                  const double *mixed, double omega, int pre, int post, int cycle,
                  int coarse_literal, double *u, const double *f) {
  if (bc_kind == BC_OPEN || bc_kind == BC_FACES) return ORC_ERR_ARG;
  Hier H;
  int st = hier_build(&H, nx, ny, nz, h);
  if (st == ORC_OK) st = hier_set_bc(&H, bc_kind, bc_value, NULL, 0, 0.0, NULL, mixed);
  if (st != ORC_OK) { hier_free(&H); return st; }
  Level *F = &H.lev[H.nlev - 1];
  load(F, F->u, u);
  load(F, F->f, f);
  Bc hom = correction_rule(&H.bcs[0], coarse_literal);
  CycleOpts o = {omega, pre, post, cycle};
  if (H.nlev == 1) coarsest(F, &H.bcs[0]);
  else multigrid(H.lev, H.nlev - 1, H.bcs, &H.bcs[H.nlev - 1], &hom, &o);
  store(F, F->u, u);
  hier_free(&H);
  return ORC_OK;
}

/* Gravitational acceleration at cell centres (Sec. 3.2.3, the cell-centred
 * source-term scheme): along each axis the two face-centred accelerations
 * -(phi_{i+1} - phi_i) / h and -(phi_i - phi_{i-1}) / h are averaged; the
 * neighbours outside the grid are ghosts from the boundary rule.  g holds the
 * three (nz, ny, nx) arrays g_x, g_y, g_z one after the other. */
int orc_op_gravity(int nx, int ny, int nz, double h, int bc_kind, double bc_value,
                   const double *faces, const double *phi, double *g) {
  OneLevel o;
  int e = one_level(&o, nx, ny, nz, h, bc_kind, bc_value, faces);
  if (e != ORC_OK) { one_free(&o); return e; }
  load(&o.L, o.L.u, phi);
  fill_ghosts(&o.L, o.L.u, &o.bc);
  const double *u = o.L.u;
  const size_t N = (size_t)nx * ny * nz;
  for (int k = 1; k <= nz; ++k)
    for (int j = 1; j <= ny; ++j)
      for (int i = 1; i <= nx; ++i) {
        const double c = u[pidx(nx, ny, i, j, k)];
        const size_t t = ((size_t)(k - 1) * ny + (j - 1)) * nx + (i - 1);
        const double xl = -(c - u[pidx(nx, ny, i - 1, j, k)]) / h;
        const double xr = -(u[pidx(nx, ny, i + 1, j, k)] - c) / h;
        const double yl = -(c - u[pidx(nx, ny, i, j - 1, k)]) / h;
        const double yr = -(u[pidx(nx, ny, i, j + 1, k)] - c) / h;
        const double zl = -(c - u[pidx(nx, ny, i, j, k - 1)]) / h;
        const double zr = -(u[pidx(nx, ny, i, j, k + 1)] - c) / h;
        g[t] = 0.5 * (xl + xr);
        g[N + t] = 0.5 * (yl + yr);
        g[2 * N + t] = 0.5 * (zl + zr);
      }
  one_free(&o);
  return ORC_OK;
}

/* The defect of Eq. (defect) on the integer grid of the mixed-precision
 * outer loop (not in the paper: its defect-correction form keeps phi and h^2 f
 * as 64-bit integers scaled by 2^S, so that the defect is exact):
 *   P' = P + round(e c)          e c the FP32 product, rounded to the nearest
 *                                integer (ties to even); P = 0 when p_in is NULL
 *   R  = F - (sum of the six neighbours of P' - 6 P')   exactly, in integers
 *   r  = fl32(R) * factor        (FP32)
 * Neighbours outside the grid follow Sec. 2.3.6 face by face (kinds[q] for
 * q = x-, x+, y-, y+, z-, z+): periodic wraps, zero gradient is the cell
 * itself, fixed b_q is B_q - P' with B_q = round(2 b_q 2^S).  Where floating
 * point decides an integer, both the rounding of e c and of 2 b_q 2^S, this
 * takes the same decision in the same precision as the CUDA kernel it checks.
 * Arrays are (nz, ny, nx) without ghosts; p_out receives P'. */
int orc_op_fx_step(int nx, int ny, int nz, const int *kinds, const double *b, double two_pow_S,
                   const long long *p_in, const float *e, float c, const long long *F,
                   long long *p_out, float factor, float *r) {
  const size_t N = (size_t)nx * ny * nz;
  long long B[6];
  for (int q = 0; q < 6; ++q) B[q] = llrint(b[q] * (2.0 * two_pow_S));
  for (size_t t = 0; t < N; ++t) {
    const float ec = e ? e[t] * c : 0.0f;
    p_out[t] = (p_in ? p_in[t] : 0) + llrintf(ec);
  }
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const size_t t = ((size_t)k * ny + j) * nx + i;
        const long long self = p_out[t];
        const int idx[3] = {i, j, k}, n[3] = {nx, ny, nz};
        long long sum = 0;
        for (int a = 0; a < 3; ++a)
          for (int side = 0; side < 2; ++side) {
            const int q = 2 * a + side;
            int m[3] = {i, j, k};
            m[a] = idx[a] + (side ? 1 : -1);
            long long v;
            if (m[a] >= 0 && m[a] < n[a]) {
              v = p_out[((size_t)m[2] * ny + m[1]) * nx + m[0]];
            } else if (kinds[q] == BC_PERIODIC) {
              m[a] = side ? 0 : n[a] - 1;
              v = p_out[((size_t)m[2] * ny + m[1]) * nx + m[0]];
            } else if (kinds[q] == BC_ZEROGRAD) {
              v = self;
            } else {
              v = B[q] - self;
            }
            sum += v;
          }
        const long long R = F[t] - (sum - 6 * self);
        r[t] = (float)R * factor;
      }
  return ORC_OK;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
