/*
 * orc.c -- plain single-threaded CPU oracle of the DIG-augmented DSMC hot path.
 *
 * TEST INFRASTRUCTURE ONLY (see orc.h).  Slow and literal on purpose: every
 * step is written out in the order the paper states it, with no blocking,
 * fusion or reordering.  Build: gcc -O2 -ffp-contract=off -fPIC -shared.
 *
 * Paper: "DIG-augmented DSMC on unstructured meshes" (arXiv 2607.08195).
 *   Sec. 2.1  DSMC: particle state (x, v, I_r; N_eff), move, NTC pair selection,
 *             VHS cross sections with VHS or VSS scattering, Borgnakke-Larsen
 *             exchange (Eq. inelastic probability), sampled moments
 *             (Eq. dsmc_temperatures).
 *   Sec. 2.2  synthetic equations (Eq. macro, Eq. synthetic_closure) and the
 *             recalibration of the particles.
 *   Sec. 3.1  exponential moving average of the summation variables
 *             (Eq. exponential_average_moments), steady cumulative average
 *             (Eq. steady_average_moments).
 *   Sec. 3.2  cell-Knudsen filter (Eq. criterion), equal-weight reconstruction
 *             (arithmetic, or the logarithmic mean named in Sec. 6) and the
 *             local accumulation state of rejected cells.
 * Where the paper names a method without giving its steps, the oracle follows
 * the published source named at that function (Bird 1994; Salmon et al. 2011;
 * Marsaglia 1972; Rocchini and Cignoni 2000; Koura and Matsumoto 1991).
 */
#include "orc.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

/* Velocity precision.  By default FP32, as the method states it: velocities,
 * rotational energies and the collision, wall and injection arithmetic in
 * single precision, with the own FP32 ln/exp below where a transcendental
 * decides (bit-identical to the CUDA path).  Built with -DORC_V64 the same
 * quantities are FP64 (libm log/pow): the FP64 reference run that states the
 * error of the FP32 path.  Positions, ray-face parameters and every sum are
 * FP64 in both builds. */
#ifdef ORC_V64
typedef double vreal;
#define VSQRT(x) sqrt(x)
#define VLN(x) log(x)
#define VEXP(x) exp(x)
#define VPOW(x, a) pow(x, a)
#define VFABS(x) fabs(x)
#define VHALF_SQRT2 0.70710678118654752
#else
typedef float vreal;
#define VSQRT(x) sqrtf(x)
#define VLN(x) orc_lnf(x)
#define VEXP(x) orc_expf(x)
#define VPOW(x, a) orc_powf(x, a)
#define VFABS(x) fabsf(x)
#define VHALF_SQRT2 0.707106781f
#endif

#define KB 1.380649e-23

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as    */
/* easy as 1, 2, 3", SC'11): ten rounds of the 4x32 Philox S-box with the     */
/* Weyl key schedule.                                                          */
/* ------------------------------------------------------------------------- */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* purposes of the random streams: key = (seed_lo, seed_hi ^ purpose << 24) */
enum { RP_INIT_POS = 1, RP_INIT_VEL = 2, RP_WALL = 3, RP_INJECT = 4, RP_COLL = 5, RP_DIR = 6,
       RP_LB = 7, RP_RECAL = 8 };

static void rng4(const orc_ctx* c, int purpose, uint32_t entity, uint32_t sub, uint32_t step,
                 uint32_t draw, uint32_t out[4]);

/* uniform in (0,1): 23 random bits, centred in their interval */
static float u01f(uint32_t w) { return ((float)(w >> 9) + 0.5f) * 0x1p-23f; }
/* uniform in (0,1) with 52 random bits */
static double u01d(uint32_t w0, uint32_t w1) {
  uint64_t k = ((uint64_t)(w0 >> 4) << 24) | (uint64_t)(w1 >> 8);
  return ((double)k + 0.5) * 0x1p-52;
}

/* ------------------------------------------------------------------------- */
/* FP32 logarithm and exponential from IEEE +,-,*,/ only, so that decisions   */
/* taken on them are reproducible on any IEEE machine.                         */
/*  ln x  = e ln 2 + 2 atanh(s),  s = (m-1)/(m+1),  m in [1/sqrt2, sqrt2)      */
/*          (atanh series to s^11)                                             */
/*  exp y = 2^k exp(r),  k = nearest integer to y/ln2, r = y - k ln2            */
/*          (Taylor series to r^7)                                             */
/*  ln 2 is split as LN2_HI + LN2_LO with LN2_HI = ln 2 truncated to 16 bits,  */
/*  so that k LN2_HI is exact for |k| <= 255 (Cody and Waite 1980).            */
/* ------------------------------------------------------------------------- */
float orc_lnf(float x) {
  uint32_t b;
  memcpy(&b, &x, 4);
  int e = (int)((b >> 23) & 0xffu) - 127;
  if (e == -127) return -87.3365448f; /* zero or subnormal: ln(2^-126) */
  uint32_t mb = (b & 0x7fffffu) | 0x3f800000u;
  float m;
  memcpy(&m, &mb, 4);
  if (m > 1.41421356f) {
    m = m * 0.5f;
    e = e + 1;
  }
  float s = (m - 1.0f) / (m + 1.0f);
  float z = s * s;
  float p = 0.0909090909f;
  p = p * z + 0.111111111f;
  p = p * z + 0.142857143f;
  p = p * z + 0.2f;
  p = p * z + 0.333333333f;
  p = p * z + 1.0f;
  float lnm = (2.0f * s) * p;
  float fe = (float)e;
  return fe * 0.693145751953125f + (lnm + fe * 1.42860677e-6f);
}

float orc_expf(float y) {
  if (y < -87.0f) return 0.0f;
  if (y > 88.0f) y = 88.0f;
  float t = y * 1.44269504f;
  int k = (int)(t >= 0.0f ? t + 0.5f : t - 0.5f);
  float fk = (float)k;
  float r = (y - fk * 0.693145751953125f) - fk * 1.42860677e-6f;
  float p = 1.98412698e-4f;
  p = p * r + 1.38888889e-3f;
  p = p * r + 8.33333333e-3f;
  p = p * r + 4.16666667e-2f;
  p = p * r + 0.166666667f;
  p = p * r + 0.5f;
  p = p * r + 1.0f;
  p = p * r + 1.0f;
  uint32_t sb = (uint32_t)(k + 127) << 23;
  float sc;
  memcpy(&sc, &sb, 4);
  return p * sc;
}

float orc_powf(float x, float a) { return orc_expf(a * orc_lnf(x)); }

/* ------------------------------------------------------------------------- */
/* context                                                                     */
/* ------------------------------------------------------------------------- */
typedef struct {
  int32_t tet, face, bc;
  vreal nrm[3], t1[3], t2[3]; /* outward unit normal and tangent basis (velocity precision) */
  /* free-stream inflow faces only */
  int32_t vtx[3];             /* the face's nodes (local order of the face) */
  double expn;                /* expected injections per step: F A dt / F_N */
  vreal s, p1, invb, sig, ut1, ut2; /* speed ratio, mixture weight, 1/beta, sqrt(kT/m), U.t1, U.t2 */
} bface_t;

#define NPHI_MAX 17
#define NMAC 20

struct orc_ctx {
  orc_config cfg;
  char err[256];
  /* mesh */
  int64_t n_tets, n_nodes;
  int32_t* nbr;      /* [4n] >=0 neighbour tet, <0: -1 - boundary-face index */
  int8_t* nbr_face;  /* [4n] local face index in the neighbour */
  double* pn;        /* [12n] outward unit normals */
  double* pd;        /* [4n]  plane offsets: n.x = d on the face */
  double* parea;     /* [4n]  face areas */
  double* vol;       /* [n] */
  double* cumvol;    /* [n] running sum of volumes */
  double* fdtv;      /* [n] F_N dt / V_c */
  double* nodes;
  int32_t* tets;
  int32_t n_bf;
  bface_t* bf;
  double* bflux;     /* [5 n_bf]: hits, momentum in (3), energy in (sum of incident minus reflected) */
  double* inj_rem;   /* [n_bf] carried fractional injection count of each inflow face */
  orc_bc* bcs;
  int32_t n_bcs;
  vreal* bc_sigma;   /* sqrt(k T / m) per bc */
  vreal* bc_U;       /* [3 n_bcs] */
  /* gas constants in the velocity precision (vreal) where the collision arithmetic uses them */
  vreal c_vhs, one_m_omega, cmax0, p_inel, lb_exp, hmr, T_init_f, sigma_init, u0f[3];
  int vss;          /* alpha != 1: VSS scattering */
  vreal inv_alpha;  /* 1 / alpha */
  int nphi;
  /* particles (sorted by cell between steps) */
  int64_t N, cap;
  double* x;
  vreal* v;
  vreal* Ir;
  int32_t* cell;
  int64_t* cstart; /* [n+1] */
  /* collision state per cell */
  vreal* cmax;
  double* rem;
  /* sampling */
  double* phi_inst;
  double* phi_ewma;
  double* phi_win;
  double* phi_cum;
  double* acc_w;   /* [n] local accumulation: samples the cell's average stands for (0: moving average) */
  int64_t n_ewma, n_win, n_cum;
  /* debug pairs */
  int64_t n_pairs, cap_pairs;
  int32_t* pr; /* 4 per pair: cell, k, i, j */
  uint8_t* pacc;
  int64_t counters[ORC_N_COUNTERS];
  int64_t step;
  /* DIG coupling */
  int64_t flux_steps;  /* DSMC steps accumulated in bflux since the last coupling */
  int64_t n_couple;    /* couplings done */
  double* cp_half;     /* [6n] M^{k+1/2} fed to the solver: rho, u(3), T_t, T_r (nondimensional) */
  double* cp_hot;      /* [12n] HoT: sigma (xx,yy,zz,xy,xz,yz), q_t (3), q_r (3) (nondimensional) */
  double* cp_new;      /* [6n] M^{k+1} */
  double* cp_own;      /* [6n] the cell's own sampled state (nondimensional) */
  float* cl_params;    /* learned-closure parameters (S12), NULL until set */
  double* cp_flag;     /* [n] 1 accepted, 2 reconstructed, 0 neither */
};

static void rng4(const orc_ctx* c, int purpose, uint32_t entity, uint32_t sub, uint32_t step,
                 uint32_t draw, uint32_t out[4]) {
  uint32_t key[2] = {(uint32_t)c->cfg.seed, (uint32_t)(c->cfg.seed >> 32) ^ ((uint32_t)purpose << 24)};
  uint32_t ctr[4] = {entity, sub, step, draw};
  orc_philox(ctr, key, out);
}

static int fail(orc_ctx* c, int code, const char* msg) {
  snprintf(c->err, sizeof c->err, "%s", msg);
  return code;
}

const char* orc_last_error(orc_ctx* c) { return c->err; }

orc_ctx* orc_create(const orc_config* cfg) {
  orc_ctx* c = (orc_ctx*)calloc(1, sizeof(orc_ctx));
  c->cfg = *cfg;
  if (c->cfg.max_cross <= 0) c->cfg.max_cross = 4096;
  c->nphi = cfg->rot_dof > 0 ? 17 : 13;
  const double m = cfg->mass, w = cfg->omega, mr = 0.5 * m;
  /* VHS: sigma_T c_r = pi d^2 (2kT_ref/(m_r c_r^2))^(w-1/2) / Gamma(5/2-w) * c_r
   *                  = C_vhs (c_r^2)^(1-w)                          (Bird 1994, eq. 4.63) */
  double cv = M_PI * cfg->d_ref * cfg->d_ref * pow(2.0 * KB * cfg->T_ref / mr, w - 0.5) / tgamma(2.5 - w);
  c->c_vhs = (vreal)cv;
  c->one_m_omega = (vreal)(1.0 - w);
  /* initial (sigma c_r)_max at c_0 = 2.5 sqrt(2 k T_init / m) */
  vreal c0sq = (vreal)(6.25 * 2.0 * KB * cfg->T_init / m);
  c->cmax0 = c->c_vhs * VPOW(c0sq, c->one_m_omega);
  /* Borgnakke-Larsen probability, Eq. inelastic_probability */
  double a = cfg->alpha;
  c->p_inel = (vreal)(a * (5.0 - 2.0 * w) * (7.0 - 2.0 * w) / (5.0 * (a + 1.0) * (a + 2.0) * cfg->Z_rot));
  /* VSS scattering law (paper Sec. 2.1) for alpha != 1; alpha = 1 is VHS */
  c->vss = a != 1.0;
  c->inv_alpha = (vreal)(1.0 / a);
  c->lb_exp = (vreal)(1.0 / (2.5 - w));
  c->hmr = (vreal)(0.5 * mr / KB); /* relative translational energy in kelvin per (m/s)^2 */
  c->T_init_f = (vreal)cfg->T_init;
  c->sigma_init = (vreal)sqrt(KB * cfg->T_init / m);
  for (int i = 0; i < 3; ++i) c->u0f[i] = (vreal)cfg->u_init[i];
  return c;
}

static void free_mesh(orc_ctx* c) {
  free(c->nbr); free(c->nbr_face); free(c->pn); free(c->pd); free(c->parea); free(c->vol); free(c->cumvol);
  free(c->cp_half); free(c->cp_hot); free(c->cp_new); free(c->cp_flag); free(c->cp_own);
  free(c->cl_params);
  free(c->fdtv); free(c->nodes); free(c->tets); free(c->bf); free(c->bflux); free(c->inj_rem); free(c->bcs);
  free(c->bc_sigma); free(c->bc_U); free(c->cstart); free(c->cmax); free(c->rem);
  free(c->phi_inst); free(c->phi_ewma); free(c->phi_win); free(c->phi_cum); free(c->acc_w);
}

void orc_destroy(orc_ctx* c) {
  if (!c) return;
  free_mesh(c);
  free(c->x); free(c->v); free(c->Ir); free(c->cell); free(c->pr); free(c->pacc);
  free(c);
}

int64_t orc_step_index(orc_ctx* c) { return c->step; }

/* ------------------------------------------------------------------------- */
/* mesh: neighbour table by matching sorted vertex triples, FP64 face planes  */
/* ------------------------------------------------------------------------- */
typedef struct { int32_t a, b, c2; int32_t tet, face; } fkey_t;

static int fkey_cmp(const void* p, const void* q) {
  const fkey_t* x = (const fkey_t*)p;
  const fkey_t* y = (const fkey_t*)q;
  if (x->a != y->a) return x->a < y->a ? -1 : 1;
  if (x->b != y->b) return x->b < y->b ? -1 : 1;
  if (x->c2 != y->c2) return x->c2 < y->c2 ? -1 : 1;
  if (x->tet != y->tet) return x->tet < y->tet ? -1 : 1;
  return x->face < y->face ? -1 : (x->face > y->face);
}

static void sort3(int32_t* v) {
  int32_t t;
  if (v[0] > v[1]) { t = v[0]; v[0] = v[1]; v[1] = t; }
  if (v[1] > v[2]) { t = v[1]; v[1] = v[2]; v[2] = t; }
  if (v[0] > v[1]) { t = v[0]; v[0] = v[1]; v[1] = t; }
}

int orc_mesh_load(orc_ctx* c, const double* nodes, int64_t n_nodes, const int32_t* tets,
                  int64_t n_tets, const int32_t* face_tag, const orc_bc* bcs, int32_t n_bcs) {
  if (n_tets <= 0 || n_nodes <= 0) return fail(c, -1, "empty mesh");
  free_mesh(c);
  const int64_t n = n_tets;
  c->n_tets = n;
  c->n_nodes = n_nodes;
  c->nodes = (double*)malloc(sizeof(double) * 3 * n_nodes);
  memcpy(c->nodes, nodes, sizeof(double) * 3 * n_nodes);
  c->tets = (int32_t*)malloc(sizeof(int32_t) * 4 * n);
  memcpy(c->tets, tets, sizeof(int32_t) * 4 * n);
  for (int64_t i = 0; i < 4 * n; ++i)
    if (tets[i] < 0 || tets[i] >= n_nodes) return fail(c, -2, "tet vertex index out of range");
  c->nbr = (int32_t*)malloc(sizeof(int32_t) * 4 * n);
  c->nbr_face = (int8_t*)malloc(4 * n);
  c->pn = (double*)malloc(sizeof(double) * 12 * n);
  c->pd = (double*)malloc(sizeof(double) * 4 * n);
  c->parea = (double*)malloc(sizeof(double) * 4 * n);
  c->vol = (double*)malloc(sizeof(double) * n);
  c->cumvol = (double*)malloc(sizeof(double) * n);
  c->fdtv = (double*)malloc(sizeof(double) * n);
  c->n_bcs = n_bcs;
  c->bcs = (orc_bc*)malloc(sizeof(orc_bc) * (n_bcs > 0 ? n_bcs : 1));
  memcpy(c->bcs, bcs, sizeof(orc_bc) * n_bcs);
  c->bc_sigma = (vreal*)malloc(sizeof(vreal) * (n_bcs > 0 ? n_bcs : 1));
  c->bc_U = (vreal*)malloc(sizeof(vreal) * 3 * (n_bcs > 0 ? n_bcs : 1));
  for (int b = 0; b < n_bcs; ++b) {
    c->bc_sigma[b] = (vreal)sqrt(KB * bcs[b].T / c->cfg.mass);
    for (int i = 0; i < 3; ++i) c->bc_U[3 * b + i] = (vreal)bcs[b].U[i];
  }

  /* volumes: V = |det(b-a, c-a, d-a)| / 6 */
  for (int64_t t = 0; t < n; ++t) {
    const double* A = nodes + 3 * tets[4 * t + 0];
    const double* B = nodes + 3 * tets[4 * t + 1];
    const double* C = nodes + 3 * tets[4 * t + 2];
    const double* D = nodes + 3 * tets[4 * t + 3];
    double u[3], v[3], w[3];
    for (int i = 0; i < 3; ++i) { u[i] = B[i] - A[i]; v[i] = C[i] - A[i]; w[i] = D[i] - A[i]; }
    double det = u[0] * (v[1] * w[2] - v[2] * w[1]) - u[1] * (v[0] * w[2] - v[2] * w[0]) +
                 u[2] * (v[0] * w[1] - v[1] * w[0]);
    double V = fabs(det) / 6.0;
    if (!(V > 0.0)) return fail(c, -2, "degenerate tetrahedron (zero volume)");
    c->vol[t] = V;
    c->cumvol[t] = (t == 0 ? 0.0 : c->cumvol[t - 1]) + V;
    c->fdtv[t] = c->cfg.F_N * c->cfg.dt / V;
  }

  /* face planes: face f is opposite local vertex f; its vertices in increasing
   * local order (a, b, c); n = (b-a) x (c-a), flipped to point away from the
   * opposite vertex, normalised; d = n . a */
  for (int64_t t = 0; t < n; ++t) {
    for (int f = 0; f < 4; ++f) {
      int lv[3], k = 0;
      for (int q = 0; q < 4; ++q)
        if (q != f) lv[k++] = q;
      const double* A = nodes + 3 * tets[4 * t + lv[0]];
      const double* B = nodes + 3 * tets[4 * t + lv[1]];
      const double* C = nodes + 3 * tets[4 * t + lv[2]];
      const double* P = nodes + 3 * tets[4 * t + f];
      double e1[3], e2[3], nn[3];
      for (int i = 0; i < 3; ++i) { e1[i] = B[i] - A[i]; e2[i] = C[i] - A[i]; }
      nn[0] = e1[1] * e2[2] - e1[2] * e2[1];
      nn[1] = e1[2] * e2[0] - e1[0] * e2[2];
      nn[2] = e1[0] * e2[1] - e1[1] * e2[0];
      double side = nn[0] * (P[0] - A[0]) + nn[1] * (P[1] - A[1]) + nn[2] * (P[2] - A[2]);
      if (side > 0.0) { nn[0] = -nn[0]; nn[1] = -nn[1]; nn[2] = -nn[2]; }
      double len = sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
      nn[0] = nn[0] / len; nn[1] = nn[1] / len; nn[2] = nn[2] / len;
      double* N = c->pn + 12 * t + 3 * f;
      N[0] = nn[0]; N[1] = nn[1]; N[2] = nn[2];
      c->pd[4 * t + f] = nn[0] * A[0] + nn[1] * A[1] + nn[2] * A[2];
      c->parea[4 * t + f] = 0.5 * len;
    }
  }

  /* neighbours: sort all faces by their vertex triple; equal triples pair up */
  fkey_t* keys = (fkey_t*)malloc(sizeof(fkey_t) * 4 * n);
  for (int64_t t = 0; t < n; ++t)
    for (int f = 0; f < 4; ++f) {
      int32_t v3[3], k = 0;
      for (int q = 0; q < 4; ++q)
        if (q != f) v3[k++] = tets[4 * t + q];
      sort3(v3);
      fkey_t* K = keys + 4 * t + f;
      K->a = v3[0]; K->b = v3[1]; K->c2 = v3[2]; K->tet = (int32_t)t; K->face = f;
    }
  qsort(keys, (size_t)(4 * n), sizeof(fkey_t), fkey_cmp);
  for (int64_t i = 0; i < 4 * n; ++i) c->nbr[i] = INT32_MIN;
  int64_t nb = 0;
  for (int64_t i = 0; i < 4 * n;) {
    int64_t j = i + 1;
    while (j < 4 * n && keys[j].a == keys[i].a && keys[j].b == keys[i].b && keys[j].c2 == keys[i].c2) ++j;
    if (j - i > 2) { free(keys); return fail(c, -2, "non-manifold face (shared by more than two tets)"); }
    if (j - i == 2) {
      fkey_t* P = keys + i;
      fkey_t* Q = keys + i + 1;
      if (face_tag[4 * P->tet + P->face] >= 0 || face_tag[4 * Q->tet + Q->face] >= 0) {
        free(keys); return fail(c, -2, "interior face carries a boundary tag");
      }
      c->nbr[4 * P->tet + P->face] = Q->tet; c->nbr_face[4 * P->tet + P->face] = (int8_t)Q->face;
      c->nbr[4 * Q->tet + Q->face] = P->tet; c->nbr_face[4 * Q->tet + Q->face] = (int8_t)P->face;
    } else {
      int32_t tag = face_tag[4 * keys[i].tet + keys[i].face];
      if (tag < 0 || tag >= n_bcs) { free(keys); return fail(c, -2, "boundary face without a valid tag"); }
      ++nb;
    }
    i = j;
  }
  free(keys);
  /* boundary faces in (tet, face) order */
  c->n_bf = (int32_t)nb;
  c->bf = (bface_t*)malloc(sizeof(bface_t) * (nb > 0 ? nb : 1));
  c->bflux = (double*)calloc(5 * (nb > 0 ? nb : 1), sizeof(double));
  c->inj_rem = (double*)calloc(nb > 0 ? nb : 1, sizeof(double));
  int32_t ib = 0;
  for (int64_t t = 0; t < n; ++t)
    for (int f = 0; f < 4; ++f) {
      if (c->nbr[4 * t + f] != INT32_MIN) continue;
      bface_t* B = c->bf + ib;
      B->tet = (int32_t)t; B->face = f; B->bc = face_tag[4 * t + f];
      const double* N = c->pn + 12 * t + 3 * f;
      /* tangent basis: t1 = normalised (a - (a.n) n) with a = e_x unless |n_x| >= 0.9
       * (then e_y); t2 = n x t1 */
      double a[3] = {1.0, 0.0, 0.0};
      if (fabs(N[0]) >= 0.9) { a[0] = 0.0; a[1] = 1.0; }
      double an = a[0] * N[0] + a[1] * N[1] + a[2] * N[2];
      double t1[3] = {a[0] - an * N[0], a[1] - an * N[1], a[2] - an * N[2]};
      double l1 = sqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
      t1[0] = t1[0] / l1; t1[1] = t1[1] / l1; t1[2] = t1[2] / l1;
      double t2[3] = {N[1] * t1[2] - N[2] * t1[1], N[2] * t1[0] - N[0] * t1[2], N[0] * t1[1] - N[1] * t1[0]};
      for (int i = 0; i < 3; ++i) { B->nrm[i] = (vreal)N[i]; B->t1[i] = (vreal)t1[i]; B->t2[i] = (vreal)t2[i]; }
      c->nbr[4 * t + f] = -1 - ib;
      c->nbr_face[4 * t + f] = (int8_t)f;
      memset(B->vtx, 0, sizeof B->vtx);
      B->expn = 0.0;
      B->s = B->p1 = B->invb = B->sig = B->ut1 = B->ut2 = 0.0f;
      const orc_bc* bc = bcs + B->bc;
      if (bc->kind == 2) {
        /* Bird (1994) eq. 4.22: one-sided number flux of a drifting Maxwellian
         * through a face with inward normal n_in = -n: F = n/(2 sqrt(pi) beta)
         * [exp(-s^2) + sqrt(pi) s (1 + erf s)], beta = sqrt(m/2kT), s = beta U.n_in */
        int k = 0;
        for (int q = 0; q < 4; ++q)
          if (q != f) B->vtx[k++] = tets[4 * t + q];
        const double* P0 = nodes + 3 * B->vtx[0];
        const double* P1 = nodes + 3 * B->vtx[1];
        const double* P2 = nodes + 3 * B->vtx[2];
        double e1[3], e2[3];
        for (int i = 0; i < 3; ++i) { e1[i] = P1[i] - P0[i]; e2[i] = P2[i] - P0[i]; }
        const double cx = e1[1] * e2[2] - e1[2] * e2[1], cy = e1[2] * e2[0] - e1[0] * e2[2],
                     cz = e1[0] * e2[1] - e1[1] * e2[0];
        const double area = 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
        const double beta = sqrt(c->cfg.mass / (2.0 * KB * bc->T));
        const double sn = -beta * (bc->U[0] * N[0] + bc->U[1] * N[1] + bc->U[2] * N[2]);
        /* 1 + erf(s) evaluated as erfc(-s): no cancellation on faces the
         * stream leaves (s << 0) */
        const double flux = bc->n / (2.0 * sqrt(M_PI) * beta) * (exp(-sn * sn) + sqrt(M_PI) * sn * erfc(-sn));
        B->expn = flux * area * c->cfg.dt / c->cfg.F_N;
        B->s = (vreal)sn;
        const double m1 = 0.5, m2 = sn > 0.0 ? sn * sqrt(M_PI) : 0.0;
        B->p1 = (vreal)(m1 / (m1 + m2));
        B->invb = (vreal)(1.0 / beta);
        B->sig = (vreal)sqrt(KB * bc->T / c->cfg.mass);
        B->ut1 = (vreal)(bc->U[0] * t1[0] + bc->U[1] * t1[1] + bc->U[2] * t1[2]);
        B->ut2 = (vreal)(bc->U[0] * t2[0] + bc->U[1] * t2[1] + bc->U[2] * t2[2]);
      }
      ++ib;
    }

  /* per-cell state */
  c->cstart = (int64_t*)calloc(n + 1, sizeof(int64_t));
  c->cmax = (vreal*)malloc(sizeof(vreal) * n);
  c->rem = (double*)calloc(n, sizeof(double));
  for (int64_t t = 0; t < n; ++t) c->cmax[t] = c->cmax0;
  c->phi_inst = (double*)calloc(NPHI_MAX * n, sizeof(double));
  c->phi_ewma = (double*)calloc(NPHI_MAX * n, sizeof(double));
  c->phi_win = (double*)calloc(NPHI_MAX * n, sizeof(double));
  c->phi_cum = (double*)calloc(NPHI_MAX * n, sizeof(double));
  c->acc_w = (double*)calloc(n, sizeof(double));
  c->n_ewma = c->n_win = c->n_cum = 0;
  return 0;
}

int orc_mesh_info(orc_ctx* c, int32_t* nbr, int8_t* nbr_face, double* normals, double* d, double* vol) {
  int64_t n = c->n_tets;
  if (nbr) memcpy(nbr, c->nbr, sizeof(int32_t) * 4 * n);
  if (nbr_face) memcpy(nbr_face, c->nbr_face, 4 * n);
  if (normals) memcpy(normals, c->pn, sizeof(double) * 12 * n);
  if (d) memcpy(d, c->pd, sizeof(double) * 4 * n);
  if (vol) memcpy(vol, c->vol, sizeof(double) * n);
  return c->n_bf;
}

/* brute-force point location: first tet whose four plane tests pass within tol */
int32_t orc_locate(orc_ctx* c, const double* x, double tol) {
  for (int64_t t = 0; t < c->n_tets; ++t) {
    int in = 1;
    for (int f = 0; f < 4 && in; ++f) {
      const double* N = c->pn + 12 * t + 3 * f;
      double s = c->pd[4 * t + f] - (N[0] * x[0] + N[1] * x[1] + N[2] * x[2]);
      if (s < -tol) in = 0;
    }
    if (in) return (int32_t)t;
  }
  return -1;
}

/* ------------------------------------------------------------------------- */
/* particle storage                                                            */
/* ------------------------------------------------------------------------- */
static void ensure_cap(orc_ctx* c, int64_t n) {
  if (n <= c->cap) return;
  int64_t cap = n + n / 2 + 16;
  c->x = (double*)realloc(c->x, sizeof(double) * 3 * cap);
  c->v = (vreal*)realloc(c->v, sizeof(vreal) * 3 * cap);
  c->Ir = (vreal*)realloc(c->Ir, sizeof(vreal) * cap);
  c->cell = (int32_t*)realloc(c->cell, sizeof(int32_t) * cap);
  c->cap = cap;
}

/* Stable counting sort of the particle array by key = 2 cell + moved, so that
 * in every cell the particles that stayed come first, in their previous
 * order, followed by the arrivals (including newly created particles), in
 * their previous order.  Particles with cell < 0 are removed.  The paper's
 * per-cell particle buckets (Listing 2) are this array cut at cstart. */
static void sort_particles(orc_ctx* c, const uint8_t* moved) {
  const int64_t n = c->n_tets, N = c->N;
  int64_t* cnt = (int64_t*)calloc(2 * n + 1, sizeof(int64_t));
  for (int64_t p = 0; p < N; ++p)
    if (c->cell[p] >= 0) cnt[2 * (int64_t)c->cell[p] + (moved ? moved[p] : 1) + 1]++;
  for (int64_t k = 0; k < 2 * n; ++k) cnt[k + 1] += cnt[k];
  int64_t M = cnt[2 * n];
  double* x = (double*)malloc(sizeof(double) * 3 * (M > 0 ? M : 1));
  vreal* v = (vreal*)malloc(sizeof(vreal) * 3 * (M > 0 ? M : 1));
  vreal* Ir = (vreal*)malloc(sizeof(vreal) * (M > 0 ? M : 1));
  int32_t* cl = (int32_t*)malloc(sizeof(int32_t) * (M > 0 ? M : 1));
  for (int64_t p = 0; p < N; ++p) {
    if (c->cell[p] < 0) continue;
    int64_t key = 2 * (int64_t)c->cell[p] + (moved ? moved[p] : 1);
    int64_t q = cnt[key]++;
    memcpy(x + 3 * q, c->x + 3 * p, 3 * sizeof(double));
    memcpy(v + 3 * q, c->v + 3 * p, 3 * sizeof(vreal));
    Ir[q] = c->Ir[p];
    cl[q] = c->cell[p];
  }
  memcpy(c->x, x, sizeof(double) * 3 * M);
  memcpy(c->v, v, sizeof(vreal) * 3 * M);
  memcpy(c->Ir, Ir, sizeof(vreal) * M);
  memcpy(c->cell, cl, sizeof(int32_t) * M);
  c->N = M;
  free(x); free(v); free(Ir); free(cl); free(cnt);
  for (int64_t t = 0; t <= n; ++t) c->cstart[t] = 0;
  for (int64_t p = 0; p < M; ++p) c->cstart[c->cell[p] + 1]++;
  for (int64_t t = 0; t < n; ++t) c->cstart[t + 1] += c->cstart[t];
}

/* Gaussian pair by Marsaglia's polar method; attempts use successive draws,
 * two attempts per Philox block. */
static uint32_t gauss2(const orc_ctx* c, int purpose, uint32_t ent, uint32_t sub, uint32_t step,
                       uint32_t draw0, vreal* g1, vreal* g2) {
  for (uint32_t d = draw0; d < draw0 + 32; ++d) {
    uint32_t w[4];
    rng4(c, purpose, ent, sub, step, d, w);
    for (int a = 0; a < 2; ++a) {
      vreal u1 = 2.0f * u01f(w[2 * a]) - 1.0f;
      vreal u2 = 2.0f * u01f(w[2 * a + 1]) - 1.0f;
      vreal s = u1 * u1 + u2 * u2;
      if (s < 1.0f && s > 0.0f) {
        vreal f = VSQRT(-2.0f * VLN(s) / s);
        *g1 = u1 * f;
        *g2 = u2 * f;
        return d + 1;
      }
    }
  }
  *g1 = 0.0f;
  *g2 = 0.0f;
  return draw0 + 32;
}

/* isotropic unit vector (Marsaglia 1972): (a,b) uniform in the unit disc,
 * e = (2a sqrt(1-s), 2b sqrt(1-s), 1-2s) with s = a^2 + b^2 */
static void unit_vector(const orc_ctx* c, int purpose, uint32_t ent, uint32_t sub, uint32_t step, vreal* e) {
  for (uint32_t d = 0; d < 32; ++d) {
    uint32_t w[4];
    rng4(c, purpose, ent, sub, step, d, w);
    for (int a = 0; a < 2; ++a) {
      vreal a1 = 2.0f * u01f(w[2 * a]) - 1.0f;
      vreal b1 = 2.0f * u01f(w[2 * a + 1]) - 1.0f;
      vreal s = a1 * a1 + b1 * b1;
      if (s < 1.0f) {
        vreal r = 2.0f * VSQRT(1.0f - s);
        e[0] = a1 * r;
        e[1] = b1 * r;
        e[2] = 1.0f - 2.0f * s;
        return;
      }
    }
  }
  e[0] = 0.0f; e[1] = 0.0f; e[2] = 1.0f;
}

/* Post-collision direction of the relative velocity under the VSS model
 * (paper Sec. 2.1; Koura & Matsumoto 1991): the impact parameter b satisfies
 * b/d = cos^alpha(chi/2) with (b/d)^2 uniform, so the deflection angle has
 * cos chi = 2 R^(1/alpha) - 1 for R uniform in (0,1); the azimuth epsilon
 * about the pre-collision direction g/|g| is uniform.  cos and sin epsilon
 * come from a uniform point (a, b) of the unit disc: (a^2 - b^2)/s and
 * 2ab/s with s = a^2 + b^2.  The new direction is
 *   e = cos chi u + sin chi (sin epsilon A + cos epsilon B)
 * with u = g/|g|, q = sqrt(u_y^2 + u_z^2), A = (q, -u_x u_y/q, -u_x u_z/q)
 * and B = (0, u_z/q, -u_y/q), an orthonormal pair perpendicular to u; when
 * q is below 1e-6 (g along x) A = (0, 1, 0) and B = (0, 0, 1).
 * Random words: draw 0 of the purpose gives R (word 0) and the first disc
 * point (words 1, 2); draws 1..31 give two points each (words 0,1 and 2,3).
 * g2 = g_x^2 + g_y^2 + g_z^2 > 0. */
static void vss_direction(const orc_ctx* c, int purpose, uint32_t ent, uint32_t sub, uint32_t step,
                          const vreal g[3], vreal g2, vreal e[3]) {
  uint32_t w[4];
  rng4(c, purpose, ent, sub, step, 0, w);
  const vreal ct = 2.0f * VPOW(u01f(w[0]), c->inv_alpha) - 1.0f;
  const vreal st = VSQRT((1.0f - ct) * (1.0f + ct));
  vreal ce = 1.0f, se = 0.0f;
  int found = 0;
  for (uint32_t d = 0; d < 32 && !found; ++d) {
    if (d > 0) rng4(c, purpose, ent, sub, step, d, w);
    /* d == 0: the point (w1, w2); d > 0: (w0, w1) then (w2, w3) */
    for (int k0 = d == 0 ? 1 : 0; k0 <= 2 && !found; k0 += 2) {
      const vreal a1 = 2.0f * u01f(w[k0]) - 1.0f;
      const vreal b1 = 2.0f * u01f(w[k0 + 1]) - 1.0f;
      const vreal s = a1 * a1 + b1 * b1;
      if (s < 1.0f && s > 0.0f) {
        ce = (a1 * a1 - b1 * b1) / s;
        se = 2.0f * a1 * b1 / s;
        found = 1;
      }
    }
  }
  const vreal gn = VSQRT(g2);
  const vreal ux = g[0] / gn, uy = g[1] / gn, uz = g[2] / gn;
  const vreal qn = VSQRT(uy * uy + uz * uz);
  if (qn > 1e-6f) {
    e[0] = ct * ux + st * se * qn;
    e[1] = ct * uy + st * (ce * uz - se * ux * uy) / qn;
    e[2] = ct * uz - st * (ce * uy + se * ux * uz) / qn;
  } else {
    e[0] = ct * ux;
    e[1] = ct * uy + st * se;
    e[2] = ct * uz + st * ce;
  }
}

int orc_vss_directions(orc_ctx* c, const float* gf, int64_t n, float* ef) {
  if (!c || (n > 0 && (!gf || !ef))) return -1;
  for (int64_t p = 0; p < n; ++p) {
    const vreal gp[3] = {gf[3 * p], gf[3 * p + 1], gf[3 * p + 2]};
    const vreal g2 = gp[0] * gp[0] + gp[1] * gp[1] + gp[2] * gp[2];
    if (!(g2 > 0.0f)) return fail(c, -1, "orc_vss_directions: zero relative velocity");
    vreal e[3];
    vss_direction(c, RP_DIR, (uint32_t)p, 0u, 0u, gp, g2, e);
    for (int i = 0; i < 3; ++i) ef[3 * p + i] = (float)e[i];
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* S0: initial state (paper Sec. 5.1: uniform equilibrium; the               */
/* initialisation step of Alg. 1)                                             */
/* ------------------------------------------------------------------------- */
int orc_particles_init(orc_ctx* c, int64_t n) {
  if (!c->vol) return fail(c, -7, "mesh not loaded");
  if (n < 0) return fail(c, -1, "negative particle count");
  ensure_cap(c, n);
  const int64_t nt = c->n_tets;
  const double Vtot = c->cumvol[nt - 1];
  for (int64_t p = 0; p < n; ++p) {
    uint32_t w[4], w2[4];
    /* cell by inverse CDF of the cumulative volume: smallest c with cum[c] > R V */
    rng4(c, RP_INIT_POS, (uint32_t)p, 0, 0, 0, w);
    double target = u01d(w[0], w[1]) * Vtot;
    int64_t lo = 0, hi = nt - 1;
    while (lo < hi) {
      int64_t mid = (lo + hi) / 2;
      if (c->cumvol[mid] > target) hi = mid; else lo = mid + 1;
    }
    int64_t t = lo;
    /* uniform point in the tet (Rocchini and Cignoni 2000, folding the unit cube) */
    rng4(c, RP_INIT_POS, (uint32_t)p, 1, 0, 0, w);
    rng4(c, RP_INIT_POS, (uint32_t)p, 2, 0, 0, w2);
    double s = u01d(w[0], w[1]), tt = u01d(w[2], w[3]), u = u01d(w2[0], w2[1]);
    if (s + tt > 1.0) { s = 1.0 - s; tt = 1.0 - tt; }
    if (tt + u > 1.0) {
      double tmp = u; u = 1.0 - s - tt; tt = 1.0 - tmp;
    } else if (s + tt + u > 1.0) {
      double tmp = u; u = s + tt + u - 1.0; s = 1.0 - tt - tmp;
    }
    const double* A = c->nodes + 3 * c->tets[4 * t + 0];
    const double* B = c->nodes + 3 * c->tets[4 * t + 1];
    const double* C = c->nodes + 3 * c->tets[4 * t + 2];
    const double* D = c->nodes + 3 * c->tets[4 * t + 3];
    for (int i = 0; i < 3; ++i)
      c->x[3 * p + i] = A[i] + s * (B[i] - A[i]) + tt * (C[i] - A[i]) + u * (D[i] - A[i]);
    /* Maxwellian velocity at T_init around u_init; rotational energy (in kelvin)
     * exponential with mean T_init (two rotational degrees of freedom) */
    vreal g[4];
    gauss2(c, RP_INIT_VEL, (uint32_t)p, 0, 0, 0, &g[0], &g[1]);
    gauss2(c, RP_INIT_VEL, (uint32_t)p, 1, 0, 0, &g[2], &g[3]);
    for (int i = 0; i < 3; ++i) c->v[3 * p + i] = c->u0f[i] + c->sigma_init * g[i];
    rng4(c, RP_INIT_VEL, (uint32_t)p, 2, 0, 0, w);
    c->Ir[p] = c->cfg.rot_dof > 0 ? -c->T_init_f * VLN(u01f(w[0])) : 0.0f;
    c->cell[p] = (int32_t)t;
  }
  c->N = n;
  sort_particles(c, NULL);
  return 0;
}

int orc_write_particles(orc_ctx* c, const double* x, const float* v, const float* Ir,
                        const int32_t* cell, int64_t n) {
  if (!c->vol) return fail(c, -7, "mesh not loaded");
  ensure_cap(c, n);
  for (int64_t p = 0; p < n; ++p)
    if (cell[p] < 0 || cell[p] >= c->n_tets) return fail(c, -1, "cell index out of range");
  memcpy(c->x, x, sizeof(double) * 3 * n);
  for (int64_t i = 0; i < 3 * n; ++i) c->v[i] = v[i];
  /* monatomic gas carries no rotational energy: I_r is ignored and reads as 0 */
  for (int64_t p = 0; p < n; ++p) c->Ir[p] = Ir && c->cfg.rot_dof > 0 ? Ir[p] : 0.0f;
  memcpy(c->cell, cell, sizeof(int32_t) * n);
  c->N = n;
  sort_particles(c, NULL);
  return 0;
}

int orc_read_particles(orc_ctx* c, double* x, float* v, float* Ir, int32_t* cell, int64_t cap, int64_t* n) {
  *n = c->N;
  if (cap < c->N) return fail(c, -3, "buffer too small");
  if (x) memcpy(x, c->x, sizeof(double) * 3 * c->N);
  if (v)
    for (int64_t i = 0; i < 3 * c->N; ++i) v[i] = (float)c->v[i];
  if (Ir)
    for (int64_t p = 0; p < c->N; ++p) Ir[p] = (float)c->Ir[p];
  if (cell) memcpy(cell, c->cell, sizeof(int32_t) * c->N);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* S2/S3: face-by-face tracking with wall interaction                         */
/* (paper Sec. 4: particles traced face by face through the cells; fully      */
/* diffuse isothermal walls, Sec. 5)                                          */
/* ------------------------------------------------------------------------- */
static double dot3(const double* n, const double* y) { return fma(n[2], y[2], fma(n[1], y[1], n[0] * y[0])); }

/* wall interaction at boundary face ib; hit counts the hits of this particle in
 * this step (it keys the random stream) */
static void wall_reflect(orc_ctx* c, int32_t ib, vreal* v, vreal* Ir, uint32_t slot, uint32_t hit, uint32_t step) {
  const bface_t* B = c->bf + ib;
  const orc_bc* bc = c->bcs + B->bc;
  vreal vin[3] = {v[0], v[1], v[2]};
  vreal Iin = *Ir;
  if (bc->kind == 1) {
    /* specular: v <- v - 2 (v.n) n */
    vreal vn = v[0] * B->nrm[0] + v[1] * B->nrm[1] + v[2] * B->nrm[2];
    vreal h = 2.0f * vn;
    for (int i = 0; i < 3; ++i) v[i] = v[i] - h * B->nrm[i];
  } else {
    /* diffuse at T_w: normal speed from the flux-weighted half-range Maxwellian,
     * tangential Gaussian components, plus the wall velocity */
    uint32_t w[4];
    rng4(c, RP_WALL, slot, hit, step, 0, w);
    vreal sg = c->bc_sigma[B->bc];
    vreal vn = sg * VSQRT(-2.0f * VLN(u01f(w[0])));
    vreal g1, g2;
    gauss2(c, RP_WALL, slot, hit, step, 1, &g1, &g2);
    vreal a = sg * g1, b = sg * g2;
    const vreal* U = c->bc_U + 3 * B->bc;
    for (int i = 0; i < 3; ++i) v[i] = ((U[i] + B->t1[i] * a) + B->t2[i] * b) - B->nrm[i] * vn;
    if (c->cfg.rot_dof > 0) *Ir = -(vreal)bc->T * VLN(u01f(w[1]));
  }
  /* wall flux bookkeeping (incident minus reflected), per boundary face */
  double* F = c->bflux + 5 * ib;
  const double m = c->cfg.mass * c->cfg.F_N;
  double ein = 0.0, eout = 0.0;
  for (int i = 0; i < 3; ++i) {
    F[1 + i] += m * ((double)vin[i] - (double)v[i]);
    ein += (double)vin[i] * vin[i];
    eout += (double)v[i] * v[i];
  }
  F[0] += 1.0;
  F[4] += 0.5 * m * (ein - eout) + c->cfg.F_N * KB * ((double)Iin - (double)*Ir);
  c->counters[ORC_C_WALL]++;
}

/* Track one particle for one time step.  Returns the final cell, or -1 if it
 * left through a free-stream / outflow face.  The algorithm (the paper gives
 * face-by-face tracking without its steps; this is the reading taken):
 *   the step's ray starts at the origin o = x with remaining time t_rem = dt
 *   and ends at e = o + v t_rem (fma per component).  Repeat: if e passes the
 *   plane tests d_f - n_f.e >= 0 of every face f other than the entry face, the
 *   particle stops at e.  Otherwise the exit face is the face f != entry with
 *   b_f = n_f.v > 0 whose hit time a_f / b_f, a_f = max(0, d_f - n_f.o), is
 *   smallest, compared without division: f precedes g iff a_f b_g < a_g b_f
 *   (ties: lowest f).  If there is none, or a_f >= t_rem b_f (the face is
 *   reached only after the step), stop at e.  Else cross: into the neighbour
 *   (entry face = its matching face; o and e unchanged), or reflect at a wall:
 *   hit time t_h = a_f / b_f, o <- o + v t_h, t_rem <- t_rem - t_h, new
 *   velocity, e <- o + v t_rem, entry face = the wall face; or leave the domain.
 * All dot products are fma(n2, y2, fma(n1, y1, n0 y0)) in FP64. */
static int32_t track_ex(orc_ctx* c, double* x, vreal* v, vreal* Ir, int32_t cell, uint32_t slot, uint32_t step,
                        double t_move, int entry0) {
  double trem = t_move;
  int entry = entry0;
  uint32_t hits = 0;
  double o[3] = {x[0], x[1], x[2]};
  double vd[3] = {(double)v[0], (double)v[1], (double)v[2]};
  double e[3];
  for (int i = 0; i < 3; ++i) e[i] = fma(vd[i], trem, o[i]);
  for (int32_t ncross = 0;; ++ncross) {
    if (ncross > c->cfg.max_cross) {
      c->counters[ORC_C_STUCK]++;
      x[0] = o[0]; x[1] = o[1]; x[2] = o[2];
      return cell;
    }
    const double* N = c->pn + 12 * (int64_t)cell;
    const double* Dp = c->pd + 4 * (int64_t)cell;
    int inside = 1;
    for (int f = 0; f < 4; ++f) {
      if (f == entry) continue;
      if (Dp[f] - dot3(N + 3 * f, e) < 0.0) inside = 0;
    }
    if (inside) {
      x[0] = e[0]; x[1] = e[1]; x[2] = e[2];
      return cell;
    }
    int best = -1;
    double ab = 0.0, bb = 1.0;
    for (int f = 0; f < 4; ++f) {
      if (f == entry) continue;
      double b = dot3(N + 3 * f, vd);
      if (!(b > 0.0)) continue;
      double a = Dp[f] - dot3(N + 3 * f, o);
      if (a < 0.0) a = 0.0;
      if (best < 0 || a * bb < ab * b) { best = f; ab = a; bb = b; }
    }
    if (best < 0 || ab >= trem * bb) {
      x[0] = e[0]; x[1] = e[1]; x[2] = e[2];
      return cell;
    }
    c->counters[ORC_C_CROSS]++;
    int32_t nb = c->nbr[4 * (int64_t)cell + best];
    if (nb >= 0) {
      entry = c->nbr_face[4 * (int64_t)cell + best];
      cell = nb;
      continue;
    }
    int32_t ib = -1 - nb;
    int kind = c->bcs[c->bf[ib].bc].kind;
    if (kind == 0 || kind == 1) {
      double th = ab / bb;
      for (int i = 0; i < 3; ++i) o[i] = fma(vd[i], th, o[i]);
      trem = trem - th;
      wall_reflect(c, ib, v, Ir, slot, hits, step);
      hits++;
      vd[0] = (double)v[0]; vd[1] = (double)v[1]; vd[2] = (double)v[2];
      for (int i = 0; i < 3; ++i) e[i] = fma(vd[i], trem, o[i]);
      entry = best;
      continue;
    }
    c->counters[ORC_C_REMOVED]++;
    return -1;
  }
}

static int32_t track(orc_ctx* c, double* x, vreal* v, vreal* Ir, int32_t cell, uint32_t slot, uint32_t step) {
  return track_ex(c, x, v, Ir, cell, slot, step, c->cfg.dt, -1);
}

int orc_track_one(orc_ctx* c, double* x, float* vf, int32_t* cell, int64_t slot, int64_t step) {
  vreal Ir = 0.0f, v[3] = {vf[0], vf[1], vf[2]};
  *cell = track(c, x, v, &Ir, *cell, (uint32_t)slot, (uint32_t)step);
  for (int i = 0; i < 3; ++i) vf[i] = (float)v[i];
  return 0;
}

/* ------------------------------------------------------------------------- */
/* S5/S6: NTC collisions (Bird 1994, Sec. 11.1) with VHS/VSS collisions and   */
/* serial Borgnakke-Larsen exchange (paper Sec. 2.1, Eq. inelastic prob.)     */
/* ------------------------------------------------------------------------- */
static void record_pair(orc_ctx* c, int32_t cell, int32_t k, int32_t i, int32_t j, int acc) {
  if (c->n_pairs >= c->cap_pairs) {
    int64_t cap = c->cap_pairs * 2 + 1024;
    c->pr = (int32_t*)realloc(c->pr, sizeof(int32_t) * 4 * cap);
    c->pacc = (uint8_t*)realloc(c->pacc, cap);
    c->cap_pairs = cap;
  }
  int32_t* r = c->pr + 4 * c->n_pairs;
  r[0] = cell; r[1] = k; r[2] = i; r[3] = j;
  c->pacc[c->n_pairs] = (uint8_t)acc;
  c->n_pairs++;
}

static void collide_cell(orc_ctx* c, int64_t cell, uint32_t step, int record) {
  const int64_t s0 = c->cstart[cell];
  const int64_t N = c->cstart[cell + 1] - s0;
  if (N < 2) return;
  /* number of candidate pairs: 1/2 N (N-1) F_N (sigma c_r)_max dt / V_c plus the
   * carried fractional remainder of this cell */
  double X = (double)N * (double)(N - 1) * 0.5 * (double)c->cmax[cell] * c->fdtv[cell] + c->rem[cell];
  double fl = floor(X);
  c->rem[cell] = X - fl;
  int64_t ncand = (int64_t)fl;
  vreal* v = c->v + 3 * s0;
  vreal* I = c->Ir + s0;
  for (int64_t k = 0; k < ncand; ++k) {
    uint32_t w[4];
    rng4(c, RP_COLL, (uint32_t)cell, (uint32_t)k, step, 0, w);
    int64_t i = (int64_t)(((uint64_t)w[0] * (uint64_t)N) >> 32);
    int64_t j = (int64_t)(((uint64_t)w[1] * (uint64_t)(N - 1)) >> 32);
    if (j >= i) j = j + 1;
    vreal g[3];
    for (int q = 0; q < 3; ++q) g[q] = v[3 * i + q] - v[3 * j + q];
    vreal g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    const vreal g2_pre = g2;
    vreal sc = g2 > 0.0f ? c->c_vhs * VPOW(g2, c->one_m_omega) : 0.0f;
    if (sc > c->cmax[cell]) c->cmax[cell] = sc;
    vreal R = u01f(w[2]);
    int acc = sc > R * c->cmax[cell];
    c->counters[ORC_C_CAND]++;
    if (record) record_pair(c, (int32_t)cell, (int32_t)k, (int32_t)i, (int32_t)j, acc);
    if (!acc) continue;
    c->counters[ORC_C_COLL]++;
    if (c->cfg.rot_dof > 0) {
      /* serial Borgnakke-Larsen: molecule i then j, each with probability
       * P_inelastic; the collision energy E_c = E_tr + I is split with
       * I'/E_c = 1 - R^(1/(5/2 - omega)) (two rotational degrees of freedom) */
      uint32_t u[4];
      rng4(c, RP_LB, (uint32_t)cell, (uint32_t)k, step, 0, u);
      vreal Etr = g2 * c->hmr;
      int64_t who[2] = {i, j};
      for (int q = 0; q < 2; ++q) {
        if (u01f(u[2 * q]) < c->p_inel) {
          vreal Ec = Etr + I[who[q]];
          vreal In = Ec * (1.0f - VPOW(u01f(u[2 * q + 1]), c->lb_exp));
          I[who[q]] = In;
          Etr = Ec - In;
          c->counters[ORC_C_LB]++;
        }
      }
      g2 = Etr / c->hmr;
    }
    vreal cr = VSQRT(g2);
    vreal e[3];
    /* VHS: isotropic; VSS: deflected from the pre-collision g */
    if (c->vss)
      vss_direction(c, RP_DIR, (uint32_t)cell, (uint32_t)k, step, g, g2_pre, e);
    else
      unit_vector(c, RP_DIR, (uint32_t)cell, (uint32_t)k, step, e);
    vreal h = 0.5f * cr;
    for (int q = 0; q < 3; ++q) {
      vreal cm = (v[3 * i + q] + v[3 * j + q]) * 0.5f;
      v[3 * i + q] = cm + h * e[q];
      v[3 * j + q] = cm - h * e[q];
    }
  }
}

/* ------------------------------------------------------------------------- */
/* S7/S8: summation variables (Eq. dsmc_temperatures, as raw sums) and their */
/* time averages (Eq. exponential_average_moments, Eq. steady_average)       */
/* Phi = [N, sum v_i (3), sum v_i^2 (3), sum vx vy, vx vz, vy vz,             */
/*        sum |v|^2 v_i (3), (diatomic) sum I, sum I v_i (3)]                 */
/* ------------------------------------------------------------------------- */
static void sample_cells(orc_ctx* c, int flags) {
  const int64_t n = c->n_tets;
  const int np = c->nphi;
  for (int64_t t = 0; t < n; ++t) {
    double ph[NPHI_MAX];
    memset(ph, 0, sizeof ph);
    for (int64_t p = c->cstart[t]; p < c->cstart[t + 1]; ++p) {
      double vx = c->v[3 * p], vy = c->v[3 * p + 1], vz = c->v[3 * p + 2];
      double vv = vx * vx + vy * vy + vz * vz;
      ph[0] += 1.0;
      ph[1] += vx; ph[2] += vy; ph[3] += vz;
      ph[4] += vx * vx; ph[5] += vy * vy; ph[6] += vz * vz;
      ph[7] += vx * vy; ph[8] += vx * vz; ph[9] += vy * vz;
      ph[10] += vv * vx; ph[11] += vv * vy; ph[12] += vv * vz;
      if (np == 17) {
        double I = c->Ir[p];
        ph[13] += I; ph[14] += I * vx; ph[15] += I * vy; ph[16] += I * vz;
      }
    }
    memcpy(c->phi_inst + NPHI_MAX * t, ph, sizeof ph);
    if (flags & ORC_EWMA) {
      /* Eq. exponential_average_moments with n_a effective samples; while
       * fewer than n_a samples exist (m <= n_a) the plain mean of all of them */
      double* E = c->phi_ewma + NPHI_MAX * t;
      const double m = (double)(c->n_ewma + 1), na = (double)c->cfg.n_a;
      double w = m < na ? m : na;
      /* a cell in the local accumulation state (Sec. 3.2) keeps every sample:
       * the running mean of its average so far (worth acc_w samples) and
       * each new step */
      if (c->cfg.local_acc && c->acc_w[t] > 0.0) {
        w = c->acc_w[t] + 1.0;
        c->acc_w[t] = w;
      }
      const double a = (w - 1.0) / w, b = 1.0 / w;
      for (int q = 0; q < np; ++q) E[q] = a * E[q] + b * ph[q];
    }
    if (flags & ORC_WINDOW) {
      double* W = c->phi_win + NPHI_MAX * t;
      for (int q = 0; q < np; ++q) W[q] += ph[q];
    }
    if (flags & ORC_CUMUL) {
      double* C = c->phi_cum + NPHI_MAX * t;
      for (int q = 0; q < np; ++q) C[q] += ph[q];
    }
  }
  if (flags & ORC_EWMA) c->n_ewma++;
  if (flags & ORC_WINDOW) c->n_win++;
  if (flags & ORC_CUMUL) c->n_cum++;
}

int orc_sample(orc_ctx* c, int32_t action) {
  const int64_t m = NPHI_MAX * c->n_tets;
  if (action & ORC_RESET_WINDOW) { memset(c->phi_win, 0, sizeof(double) * m); c->n_win = 0; }
  if (action & ORC_RESET_CUMUL) { memset(c->phi_cum, 0, sizeof(double) * m); c->n_cum = 0; }
  if (action & ORC_RESET_EWMA) {
    memset(c->phi_ewma, 0, sizeof(double) * m);
    memset(c->acc_w, 0, sizeof(double) * c->n_tets);
    c->n_ewma = 0;
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* S4: free-stream injection.  Per inflow face and step: N = floor(E + r),    */
/* r <- E + r - N (E = F A dt / F_N).  Each new particle: uniform point on    */
/* the face; tangential velocity U_t + N(0, kT/m); inward normal speed from    */
/* the drifting flux distribution g(z) ~ z exp(-(z-s)^2), z > 0 (z = beta v_n)*/
/* sampled by acceptance-rejection (below); then it moves for a uniform       */
/* fraction of dt from the face into the domain.                               */
/*   s <= 0: z = sqrt(-ln R) (density z exp(-z^2)), accept with exp(2 s z).   */
/*   s > 0:  dominating function (z-s)^+ e^{-(z-s)^2} + s e^{-(z-s)^2} on all */
/*           z, component masses 1/2 and s sqrt(pi): z = s + sqrt(-ln R) from */
/*           the first (always accepted), or z = s + N(0,1/2) from the second,*/
/*           rejected if z <= 0 and accepted with z/s if z < s -- the ratio   */
/*           g / dominating function (g = 0 for z <= 0).                      */
/* Random stream: entity = boundary face, sub = k, draw 0 position, draw 1    */
/* fraction of dt, draws 2.. tangential Gaussian pair, then normal speed      */
/* attempts, then (diatomic) the rotational energy.                            */
/* ------------------------------------------------------------------------- */
static vreal inflow_normal_speed(const orc_ctx* c, const bface_t* B, uint32_t ib, uint32_t k, uint32_t step,
                                 uint32_t* draw) {
  const vreal s = B->s;
  for (int att = 0; att < 64; ++att) {
    uint32_t w[4];
    rng4(c, RP_INJECT, ib, k, step, (*draw)++, w);
    if (s <= 0.0f) {
      vreal z = VSQRT(-VLN(u01f(w[0])));
      if (u01f(w[1]) < VEXP(2.0f * s * z)) return z;
    } else if (u01f(w[0]) < B->p1) {
      return s + VSQRT(-VLN(u01f(w[1])));
    } else {
      /* the second component's Gaussian is drawn to completion (polar method
       * over the following draws) before the acceptance test */
      vreal g1, g2;
      *draw = gauss2(c, RP_INJECT, ib, k, step, *draw, &g1, &g2);
      vreal z = s + g1 * VHALF_SQRT2;
      if (z > 0.0f && (z >= s || u01f(w[3]) * s < z)) return z;
    }
  }
  return s > 0.0f ? s : 0.5f;
}

static void inject(orc_ctx* c, uint32_t step, uint8_t** moved, int64_t* cap_moved) {
  for (int32_t ib = 0; ib < c->n_bf; ++ib) {
    const bface_t* B = c->bf + ib;
    if (c->bcs[B->bc].kind != 2) continue;
    double X = B->expn + c->inj_rem[ib];
    double fl = floor(X);
    c->inj_rem[ib] = X - fl;
    const int64_t n = (int64_t)fl;
    for (int64_t k = 0; k < n; ++k) {
      const int64_t p = c->N;
      ensure_cap(c, p + 1);
      if (p + 1 > *cap_moved) {
        *cap_moved = 2 * (p + 1);
        *moved = (uint8_t*)realloc(*moved, (size_t)*cap_moved);
      }
      uint32_t w[4];
      rng4(c, RP_INJECT, (uint32_t)ib, (uint32_t)k, step, 0, w);
      double r1 = u01d(w[0], w[1]), r2 = u01d(w[2], w[3]);
      if (r1 + r2 > 1.0) { r1 = 1.0 - r1; r2 = 1.0 - r2; }
      const double* A = c->nodes + 3 * B->vtx[0];
      const double* P1 = c->nodes + 3 * B->vtx[1];
      const double* P2 = c->nodes + 3 * B->vtx[2];
      double* x = c->x + 3 * p;
      for (int i = 0; i < 3; ++i) x[i] = A[i] + r1 * (P1[i] - A[i]) + r2 * (P2[i] - A[i]);
      rng4(c, RP_INJECT, (uint32_t)ib, (uint32_t)k, step, 1, w);
      const double tfrac = u01d(w[0], w[1]);
      vreal g1, g2;
      uint32_t draw = gauss2(c, RP_INJECT, (uint32_t)ib, (uint32_t)k, step, 2, &g1, &g2);
      const vreal vn = inflow_normal_speed(c, B, (uint32_t)ib, (uint32_t)k, step, &draw) * B->invb;
      const vreal a = B->ut1 + B->sig * g1, b = B->ut2 + B->sig * g2;
      vreal* v = c->v + 3 * p;
      for (int i = 0; i < 3; ++i) v[i] = (B->t1[i] * a + B->t2[i] * b) - B->nrm[i] * vn;
      c->Ir[p] = 0.0f;
      if (c->cfg.rot_dof > 0) {
        rng4(c, RP_INJECT, (uint32_t)ib, (uint32_t)k, step, draw, w);
        c->Ir[p] = -(vreal)c->bcs[B->bc].T * VLN(u01f(w[0]));
      }
      c->N = p + 1;
      c->counters[ORC_C_INJECTED]++;
      c->cell[p] = track_ex(c, x, v, c->Ir + p, B->tet, (uint32_t)p, step, tfrac * c->cfg.dt, B->face);
      (*moved)[p] = 1;
    }
  }
}

/* ------------------------------------------------------------------------- */
/* one DSMC time step: move (with walls / outflow), sort, collide, sample     */
/* ------------------------------------------------------------------------- */
int orc_dsmc_step(orc_ctx* c, int32_t n_steps, int32_t flags) {
  if (!c->vol) return fail(c, -7, "mesh not loaded");
  int record = (flags & ORC_RECORD_PAIRS) != 0;
  for (int32_t s = 0; s < n_steps; ++s) {
    c->step += 1;
    const uint32_t step = (uint32_t)c->step;
    c->n_pairs = 0;
    const int64_t N = c->N;
    int64_t cap_moved = N + 1024;
    uint8_t* moved = (uint8_t*)malloc((size_t)cap_moved);
    for (int64_t p = 0; p < N; ++p) {
      int32_t old = c->cell[p];
      int32_t nc = track(c, c->x + 3 * p, c->v + 3 * p, c->Ir + p, old, (uint32_t)p, step);
      c->cell[p] = nc;
      moved[p] = (uint8_t)(nc != old);
    }
    inject(c, step, &moved, &cap_moved);
    sort_particles(c, moved);
    free(moved);
    for (int64_t t = 0; t < c->n_tets; ++t) collide_cell(c, t, step, record);
    sample_cells(c, flags & (ORC_EWMA | ORC_WINDOW | ORC_CUMUL));
    c->counters[ORC_C_STEPS]++;
    c->flux_steps++;
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* read-out: raw summation variables, or the macroscopic moments derived from */
/* averaged sums (Eq. dsmc_temperatures, dimensional):                        */
/* [0] mean N, [1] rho, [2..4] u, [5] T_t, [6] T_r, [7] T, [8..13] sigma      */
/* (xx,yy,zz,xy,xz,yz), [14..16] q_t, [17..19] q_r                            */
/* ------------------------------------------------------------------------- */
static void derive_macro(const orc_ctx* c, const double* ph, double V, double* M) {
  const double m = c->cfg.mass, FN = c->cfg.F_N;
  memset(M, 0, sizeof(double) * NMAC);
  double N = ph[0];
  M[0] = N;
  if (!(N > 0.0)) return;
  double u[3] = {ph[1] / N, ph[2] / N, ph[3] / N};
  double vv[3][3];
  vv[0][0] = ph[4] / N; vv[1][1] = ph[5] / N; vv[2][2] = ph[6] / N;
  vv[0][1] = vv[1][0] = ph[7] / N; vv[0][2] = vv[2][0] = ph[8] / N; vv[1][2] = vv[2][1] = ph[9] / N;
  double cc[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) cc[i][j] = vv[i][j] - u[i] * u[j];
  double tr = cc[0][0] + cc[1][1] + cc[2][2];
  double v2 = vv[0][0] + vv[1][1] + vv[2][2];
  double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  double rho = m * FN * N / V;
  M[1] = rho;
  M[2] = u[0]; M[3] = u[1]; M[4] = u[2];
  double Tt = m * tr / (3.0 * KB);
  M[5] = Tt;
  int dr = c->cfg.rot_dof;
  double Tr = 0.0;
  if (dr > 0) Tr = 2.0 * (ph[13] / N) / dr;
  M[6] = Tr;
  M[7] = (3.0 * Tt + dr * Tr) / (3.0 + dr);
  M[8] = rho * (cc[0][0] - tr / 3.0);
  M[9] = rho * (cc[1][1] - tr / 3.0);
  M[10] = rho * (cc[2][2] - tr / 3.0);
  M[11] = rho * cc[0][1];
  M[12] = rho * cc[0][2];
  M[13] = rho * cc[1][2];
  for (int i = 0; i < 3; ++i) {
    /* <c_i c^2> = <v_i v^2> - 2 u_j <v_i v_j> - u_i <v^2> + 2 u_i |u|^2 */
    double uj = u[0] * vv[i][0] + u[1] * vv[i][1] + u[2] * vv[i][2];
    double c3 = ph[10 + i] / N - 2.0 * uj - u[i] * v2 + 2.0 * u[i] * uu;
    M[14 + i] = 0.5 * rho * c3;
    if (dr > 0) M[17 + i] = (FN * N / V) * KB * (ph[14 + i] / N - u[i] * (ph[13] / N));
  }
}

int orc_read_moments(orc_ctx* c, int32_t which, double* out, int64_t cap) {
  const int64_t n = c->n_tets;
  int base = which & 15;
  const double* src = base == ORC_PHI_INST ? c->phi_inst
                    : base == ORC_PHI_EWMA ? c->phi_ewma
                    : base == ORC_PHI_WINDOW ? c->phi_win : c->phi_cum;
  if (!(which & ORC_MACRO)) {
    if (cap < NPHI_MAX * n) return fail(c, -3, "buffer too small");
    memcpy(out, src, sizeof(double) * NPHI_MAX * n);
    return 0;
  }
  if (cap < NMAC * n) return fail(c, -3, "buffer too small");
  double cnt = base == ORC_PHI_WINDOW ? (double)c->n_win : base == ORC_PHI_CUM ? (double)c->n_cum : 1.0;
  for (int64_t t = 0; t < n; ++t) {
    double ph[NPHI_MAX];
    for (int q = 0; q < NPHI_MAX; ++q) ph[q] = cnt > 0 ? src[NPHI_MAX * t + q] / cnt : 0.0;
    derive_macro(c, ph, c->vol[t], out + NMAC * t);
  }
  return 0;
}

int orc_read_pairs(orc_ctx* c, int32_t* cell, int32_t* k, int32_t* i, int32_t* j, uint8_t* acc,
                   int64_t cap, int64_t* n) {
  *n = c->n_pairs;
  if (cap < c->n_pairs) return fail(c, -3, "buffer too small");
  for (int64_t q = 0; q < c->n_pairs; ++q) {
    cell[q] = c->pr[4 * q]; k[q] = c->pr[4 * q + 1]; i[q] = c->pr[4 * q + 2]; j[q] = c->pr[4 * q + 3];
    acc[q] = c->pacc[q];
  }
  return 0;
}

int orc_read_counters(orc_ctx* c, int64_t* out, int32_t n) {
  for (int32_t q = 0; q < n && q < ORC_N_COUNTERS; ++q) out[q] = c->counters[q];
  return 0;
}

int orc_cell_state(orc_ctx* c, float* cmax, double* rem, int32_t write) {
  const int64_t n = c->n_tets;
  if (write) {
    if (cmax)
      for (int64_t t = 0; t < n; ++t) c->cmax[t] = cmax[t];
    if (rem) memcpy(c->rem, rem, sizeof(double) * n);
  } else {
    if (cmax)
      for (int64_t t = 0; t < n; ++t) cmax[t] = (float)c->cmax[t];
    if (rem) memcpy(rem, c->rem, sizeof(double) * n);
  }
  return 0;
}

int orc_wall_flux(orc_ctx* c, double* out, int64_t cap, int64_t* n_bfaces) {
  *n_bfaces = c->n_bf;
  if (cap < 5 * (int64_t)c->n_bf) return fail(c, -3, "buffer too small");
  memcpy(out, c->bflux, sizeof(double) * 5 * c->n_bf);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* standalone stable counting sort by cell                                     */
/* ------------------------------------------------------------------------- */
int orc_sort_by_cell(const int32_t* cell, int64_t n, int32_t n_cells, int32_t* cell_start, int32_t* order) {
  if (n < 0 || n_cells <= 0) return -1;
  for (int32_t c = 0; c <= n_cells; ++c) cell_start[c] = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (cell[i] < -1 || cell[i] >= n_cells) return -1;
    if (cell[i] >= 0) cell_start[cell[i] + 1]++;
  }
  for (int32_t c = 0; c < n_cells; ++c) cell_start[c + 1] += cell_start[c];
  int32_t* cur = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_cells);
  for (int32_t c = 0; c < n_cells; ++c) cur[c] = cell_start[c];
  for (int64_t i = 0; i < n; ++i)
    if (cell[i] >= 0) order[cur[cell[i]]++] = (int32_t)i;
  free(cur);
  return 0;
}

/* ========================================================================= */
/* DIG coupling (paper Sec. 3, Alg. 1): S9 HoT extraction and reliability    */
/* filter, S10 synthetic-equation solve, S11 particle recalibration.         */
/* Nondimensional variables (Sec. 2.2): lengths / L0, density / (m n0),      */
/* temperature / T0, velocity / sqrt(R T0), R = k/m; then p = rho T_t,       */
/* mu = Kn sqrt(2/pi) T_t^omega (from the paper's Kn definition), stress /   */
/* (rho0 R T0), heat flux / (rho0 (R T0)^{3/2}).                              */
/* ========================================================================= */
typedef struct {
  double L0, T0, rho0, c0, Kn, omega, gam, dr, Zr;
} nd_t;

static nd_t nondim(const orc_ctx* c) {
  nd_t d;
  d.L0 = c->cfg.L_ref;
  d.T0 = c->cfg.T_init;
  d.rho0 = c->cfg.mass * c->cfg.n_init;
  d.c0 = sqrt(KB / c->cfg.mass * d.T0);
  d.Kn = c->cfg.Kn;
  d.omega = c->cfg.omega;
  d.dr = (double)c->cfg.rot_dof;
  d.gam = (5.0 + d.dr) / (3.0 + d.dr);
  d.Zr = c->cfg.Z_rot;
  return d;
}

/* viscosity and conductivities (Sec. 2.2, NSF relations; the heat-flux
 * relaxation matrix is not given: kappa_t = 15/4 mu, kappa_r = 1.32 mu) */
static double mu_nd(const nd_t* d, double Tt) { return d->Kn * sqrt(2.0 / M_PI) * pow(Tt > 1e-6 ? Tt : 1e-6, d->omega); }

/* boundary values of u, T_t, T_r at boundary face ib (walls: wall values;
 * open faces: free stream) */
/* values of u (3), T_t and T_r at a boundary face with outward unit normal N,
 * seen from a cell with primitives Pc: a diffuse wall or an inflow face gives
 * its own velocity and temperature; a specular wall the cell's velocity
 * without its normal component and the cell's temperatures (slip, adiabatic);
 * an outflow face the cell's own values */
static void bc_values(const orc_ctx* c, const nd_t* d, int32_t ib, const double* Pc, const double* N, double* phi) {
  const orc_bc* b = c->bcs + c->bf[ib].bc;
  if (b->kind == 1) {
    const double un = Pc[1] * N[0] + Pc[2] * N[1] + Pc[3] * N[2];
    for (int i = 0; i < 3; ++i) phi[i] = Pc[1 + i] - un * N[i];
    phi[3] = Pc[4];
    phi[4] = Pc[5];
  } else if (b->kind == 3) {
    for (int q = 0; q < 5; ++q) phi[q] = Pc[1 + q];
  } else {
    for (int i = 0; i < 3; ++i) phi[i] = b->U[i] / d->c0;
    phi[3] = b->T / d->T0;
    phi[4] = phi[3];
  }
}

/* Least-squares gradients of u (3) and T_t, T_r at every cell: the gradient
 * G minimising sum_f |phi_f - phi_c - G . d_f|^2 over the four faces, with
 * d_f = x_f - x_c (nondimensional), x_f the neighbour's centroid across an
 * interior face and the face centroid at a boundary face, where phi_f is the
 * boundary value; G = (sum_f d_f d_f^T)^-1 sum_f d_f (phi_f - phi_c).  Exact
 * for linear fields on any tetrahedron.  prim[6n]: rho, u(3), T_t, T_r. */
static void tet_centroid(const orc_ctx* c, int64_t t, double s, double* x) {
  for (int i = 0; i < 3; ++i) {
    double a = 0.0;
    for (int v = 0; v < 4; ++v) a += c->nodes[3 * (int64_t)c->tets[4 * t + v] + i];
    x[i] = 0.25 * a * s;
  }
}

static void gradients(const orc_ctx* c, const nd_t* d, const double* prim, double* grad /* [15n] */) {
  const int64_t n = c->n_tets;
  const double s = 1.0 / d->L0;
  for (int64_t t = 0; t < n; ++t) {
    const double* Pc = prim + 6 * t;
    double xc[3], M[3][3], b[15];
    memset(M, 0, sizeof M);
    memset(b, 0, sizeof b);
    tet_centroid(c, t, s, xc);
    for (int f = 0; f < 4; ++f) {
      const int32_t nb = c->nbr[4 * t + f];
      double xf[3], phi[5];
      if (nb >= 0) {
        tet_centroid(c, nb, s, xf);
        for (int q = 0; q < 5; ++q) phi[q] = prim[6 * (int64_t)nb + 1 + q];
      } else {
        /* centroid of face f: the three vertices other than vertex f */
        for (int i = 0; i < 3; ++i) {
          double a = 0.0;
          for (int v = 0; v < 4; ++v)
            if (v != f) a += c->nodes[3 * (int64_t)c->tets[4 * t + v] + i];
          xf[i] = a / 3.0 * s;
        }
        bc_values(c, d, -1 - nb, Pc, c->pn + 12 * t + 3 * f, phi);
      }
      const double df[3] = {xf[0] - xc[0], xf[1] - xc[1], xf[2] - xc[2]};
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[i][j] += df[i] * df[j];
      for (int q = 0; q < 5; ++q)
        for (int i = 0; i < 3; ++i) b[3 * q + i] += df[i] * (phi[q] - Pc[1 + q]);
    }
    /* inverse of the symmetric 3x3 matrix M by cofactors */
    double A[3][3];
    A[0][0] = M[1][1] * M[2][2] - M[1][2] * M[2][1];
    A[0][1] = M[0][2] * M[2][1] - M[0][1] * M[2][2];
    A[0][2] = M[0][1] * M[1][2] - M[0][2] * M[1][1];
    A[1][0] = M[1][2] * M[2][0] - M[1][0] * M[2][2];
    A[1][1] = M[0][0] * M[2][2] - M[0][2] * M[2][0];
    A[1][2] = M[0][2] * M[1][0] - M[0][0] * M[1][2];
    A[2][0] = M[1][0] * M[2][1] - M[1][1] * M[2][0];
    A[2][1] = M[0][1] * M[2][0] - M[0][0] * M[2][1];
    A[2][2] = M[0][0] * M[1][1] - M[0][1] * M[1][0];
    const double det = M[0][0] * A[0][0] + M[0][1] * A[1][0] + M[0][2] * A[2][0];
    for (int q = 0; q < 5; ++q)
      for (int i = 0; i < 3; ++i)
        grad[15 * t + 3 * q + i] = (A[i][0] * b[3 * q] + A[i][1] * b[3 * q + 1] + A[i][2] * b[3 * q + 2]) / det;
  }
}

/* NSF stress (6) and heat fluxes (3 + 3) of one cell from its primitives and gradients */
static void nsf(const nd_t* d, const double* P, const double* G, double* sig, double* qt, double* qr) {
  const double mu = mu_nd(d, P[4]);
  /* G[3q + i] = d phi_q / d x_i ; phi_0..2 = u_x,u_y,u_z */
  const double div = G[0] + G[4] + G[8];
  sig[0] = -mu * (2.0 * G[0] - 2.0 / 3.0 * div);
  sig[1] = -mu * (2.0 * G[4] - 2.0 / 3.0 * div);
  sig[2] = -mu * (2.0 * G[8] - 2.0 / 3.0 * div);
  sig[3] = -mu * (G[1] + G[3]);
  sig[4] = -mu * (G[2] + G[6]);
  sig[5] = -mu * (G[5] + G[7]);
  const double kt = 3.75 * mu, kr = 1.32 * mu;
  for (int i = 0; i < 3; ++i) {
    qt[i] = -kt * G[9 + i];
    qr[i] = d->dr > 0 ? -kr * G[12 + i] : 0.0;
  }
}

/* S9 first half: from summation variables phi (sums over cnt steps; cnt = 1
 * for the moving average) the cell's own nondimensional state own[6n] (rho,
 * u(3), T_t, T_r), its mean particle count nbar[n] and HoT[12n] = sampled
 * stress / heat flux minus their NSF values at the gradients of that state
 * (Sec. 3.1, Eq. hot_extraction) */
static void sampled_hot(orc_ctx* c, const nd_t* d, const double* phi, double cnt, double* own, double* H,
                        double* nbar) {
  const int64_t n = c->n_tets;
  double* grad = (double*)malloc(sizeof(double) * 15 * n);
  double* sdsmc = (double*)malloc(sizeof(double) * 12 * n);
  for (int64_t t = 0; t < n; ++t) {
    double ph[NPHI_MAX], M[NMAC];
    for (int q = 0; q < NPHI_MAX; ++q)
      ph[q] = cnt == 1.0 ? phi[NPHI_MAX * t + q] : cnt > 0 ? phi[NPHI_MAX * t + q] / cnt : 0.0;
    derive_macro(c, ph, c->vol[t], M);
    nbar[t] = M[0];
    double* o = own + 6 * t;
    o[0] = M[1] / d->rho0;
    o[1] = M[2] / d->c0; o[2] = M[3] / d->c0; o[3] = M[4] / d->c0;
    o[4] = M[5] / d->T0;
    o[5] = d->dr > 0 ? M[6] / d->T0 : o[4];
    const double ss = d->rho0 * d->c0 * d->c0, qs = ss * d->c0;
    for (int q = 0; q < 6; ++q) sdsmc[12 * t + q] = M[8 + q] / ss;
    for (int q = 0; q < 3; ++q) {
      sdsmc[12 * t + 6 + q] = M[14 + q] / qs;
      sdsmc[12 * t + 9 + q] = M[17 + q] / qs;
    }
  }
  gradients(c, d, own, grad);
  for (int64_t t = 0; t < n; ++t) {
    double sig[6], qt[3], qr[3];
    nsf(d, own + 6 * t, grad + 15 * t, sig, qt, qr);
    double* h = H + 12 * t;
    for (int q = 0; q < 6; ++q) h[q] = sdsmc[12 * t + q] - sig[q];
    for (int q = 0; q < 3; ++q) {
      h[6 + q] = sdsmc[12 * t + 6 + q] - qt[q];
      h[9 + q] = sdsmc[12 * t + 9 + q] - qr[q];
    }
  }
  free(grad); free(sdsmc);
}

/* S12 inputs: 13 features per cell from summation variables phi over cnt
 * steps -- rho, u(3), T_t (nondimensional) and the traceless HoT stress
 * (xx, yy, xy, xz, yz) over rho T_t and translational HoT heat flux over
 * rho T_t^{3/2} (i.e. sigma / (rho k T / m), q / (rho (k T / m)^{3/2}) in SI).
 * A cell without particles, or with a non-positive or non-finite state, gets
 * a zero row and valid[t] = 0.  own[6n] receives the cells' states. */
static void closure_inputs(orc_ctx* c, const nd_t* d, const double* phi, double cnt, float* X, double* own,
                           uint8_t* valid) {
  const int64_t n = c->n_tets;
  double* H = (double*)malloc(sizeof(double) * 12 * n);
  double* nbar = (double*)malloc(sizeof(double) * n);
  sampled_hot(c, d, phi, cnt, own, H, nbar);
  for (int64_t t = 0; t < n; ++t) {
    const double* o = own + 6 * t;
    const double* h = H + 12 * t;
    int ok = cnt > 0 && nbar[t] > 0.0 && o[0] > 0.0 && o[4] > 0.0;
    double f[13];
    if (ok) {
      const double s = o[0] * o[4], qn = s * sqrt(o[4]);
      f[0] = o[0]; f[1] = o[1]; f[2] = o[2]; f[3] = o[3]; f[4] = o[4];
      f[5] = h[0] / s; f[6] = h[1] / s; f[7] = h[3] / s; f[8] = h[4] / s; f[9] = h[5] / s;
      f[10] = h[6] / qn; f[11] = h[7] / qn; f[12] = h[8] / qn;
      for (int k = 0; k < 13 && ok; ++k) ok = isfinite(f[k]) && isfinite((float)f[k]);
    }
    for (int k = 0; k < 13; ++k) X[13 * t + k] = ok ? (float)f[k] : 0.0f;
    if (valid) valid[t] = (uint8_t)ok;
  }
  free(H); free(nbar);
}

static const double* phi_select(const orc_ctx* c, int32_t which, double* cnt) {
  *cnt = which == ORC_PHI_WINDOW ? (double)c->n_win : which == ORC_PHI_CUM ? (double)c->n_cum : 1.0;
  return which == ORC_PHI_INST ? c->phi_inst : which == ORC_PHI_EWMA ? c->phi_ewma
       : which == ORC_PHI_WINDOW ? c->phi_win : c->phi_cum;
}

/* S12 in the coupling: the learned closure evaluated on the coupling
 * window's features replaces the translational HoT (sigma, q_t) of every cell
 * whose features are valid and whose prediction is finite and within
 * ORC_CLOSURE_YMAX; the other cells keep the sampled HoT (the fallback).
 * sigma_zz = -(sigma_xx + sigma_yy); q_r keeps its sampled value. */
static int64_t closure_apply(orc_ctx* c, const nd_t* d) {
  const int64_t n = c->n_tets;
  float* X = (float*)malloc(sizeof(float) * 13 * n);
  double* Y = (double*)malloc(sizeof(double) * 8 * n);
  double* own = (double*)malloc(sizeof(double) * 6 * n);
  uint8_t* valid = (uint8_t*)malloc(n);
  closure_inputs(c, d, c->phi_win, (double)c->n_win, X, own, valid);
  orc_mlp_forward(c->cl_params, X, n, 1, Y);
  int64_t used = 0;
  for (int64_t t = 0; t < n; ++t) {
    const double* y = Y + 8 * t;
    int ok = valid[t];
    for (int k = 0; k < 8 && ok; ++k) ok = isfinite(y[k]) && fabs(y[k]) <= ORC_CLOSURE_YMAX;
    if (!ok) continue;
    const double rho = own[6 * t], T = own[6 * t + 4];
    const double s = rho * T, qn = s * sqrt(T);
    double* h = c->cp_hot + 12 * t;
    h[0] = y[0] * s;
    h[1] = y[1] * s;
    h[2] = -(h[0] + h[1]);
    h[3] = y[2] * s;
    h[4] = y[3] * s;
    h[5] = y[4] * s;
    for (int q = 0; q < 3; ++q) h[6 + q] = y[5 + q] * qn;
    used++;
  }
  free(X); free(Y); free(own); free(valid);
  return used;
}

/* Reconstruction of cell t from its available face neighbours, every
 * neighbour with the same weight (Sec. 3.2): the arithmetic mean of state and
 * HoT; with recon = 1 the density and the temperatures take the logarithmic
 * (geometric) mean exp(mean ln) instead -- the log-mean reconstruction that
 * the paper's conclusions (Sec. 6) name -- when all contributing values are
 * positive (the arithmetic mean otherwise).  Returns the number of
 * contributing neighbours (0: nothing written). */
static int neighbour_mean(orc_ctx* c, int64_t t, const uint8_t* avail) {
  static const int lq[3] = {0, 4, 5};
  double acc[18], lg[3] = {0.0, 0.0, 0.0};
  int pos[3] = {1, 1, 1};
  memset(acc, 0, sizeof acc);
  int cnt = 0;
  for (int f = 0; f < 4; ++f) {
    const int32_t nb = c->nbr[4 * t + f];
    if (nb < 0 || !avail[nb]) continue;
    const double* h = c->cp_half + 6 * (int64_t)nb;
    for (int q = 0; q < 6; ++q) acc[q] += h[q];
    for (int q = 0; q < 12; ++q) acc[6 + q] += c->cp_hot[12 * (int64_t)nb + q];
    for (int k = 0; k < 3; ++k) {
      if (h[lq[k]] > 0.0)
        lg[k] += log(h[lq[k]]);
      else
        pos[k] = 0;
    }
    cnt++;
  }
  if (cnt == 0) return 0;
  for (int q = 0; q < 6; ++q) c->cp_half[6 * t + q] = acc[q] / cnt;
  for (int q = 0; q < 12; ++q) c->cp_hot[12 * t + q] = acc[6 + q] / cnt;
  if (c->cfg.recon == 1)
    for (int k = 0; k < 3; ++k)
      if (pos[k]) c->cp_half[6 * t + lq[k]] = exp(lg[k] / cnt);
  return cnt;
}

/* S9: M^{k+1/2}, HoT and the reliability filter with neighbour reconstruction */
static void extract_hot(orc_ctx* c, const nd_t* d, int64_t* n_rej, int64_t* n_rec, int64_t* n_learned) {
  const int64_t n = c->n_tets;
  double* nbar = (double*)malloc(sizeof(double) * n);
  sampled_hot(c, d, c->phi_ewma, 1.0, c->cp_own, c->cp_hot, nbar);
  uint8_t* avail = (uint8_t*)calloc(n, 1);
  *n_rej = 0;
  for (int64_t t = 0; t < n; ++t) {
    const double* P = c->cp_own + 6 * t;
    const double* H = c->cp_hot + 12 * t;
    memcpy(c->cp_half + 6 * t, P, 6 * sizeof(double));
    /* local cell Knudsen number (Eq. cell_kn_stability) */
    const double V = c->vol[t] / (d->L0 * d->L0 * d->L0);
    const double dc = 2.0 * cbrt(3.0 * V / (4.0 * M_PI));
    /* a state needs at least two particles on average to have a temperature */
    int ok = nbar[t] >= 2.0 && P[0] > 0.0 && P[4] > 0.0;
    for (int q = 0; q < 6 && ok; ++q) ok = isfinite(P[q]);
    for (int q = 0; q < 12 && ok; ++q) ok = isfinite(H[q]);
    if (ok) {
      const double lam = d->Kn * pow(P[4], d->omega - 0.5) / P[0];
      ok = lam / dc <= c->cfg.KnD_max;
    }
    avail[t] = (uint8_t)ok;
    c->cp_flag[t] = ok ? 1.0 : 0.0;
    if (!ok) (*n_rej)++;
    /* local accumulation state (Sec. 3.2): a rejected cell stops forgetting;
     * its moving average so far counts as the min(m, n_a) samples it stands
     * for.  An accepted cell returns to the moving average. */
    if (c->cfg.local_acc) {
      if (ok)
        c->acc_w[t] = 0.0;
      else if (c->acc_w[t] == 0.0)
        c->acc_w[t] = (double)(c->n_ewma < c->cfg.n_a ? c->n_ewma : c->cfg.n_a);
    }
  }
  *n_learned = c->cfg.closure && c->cl_params ? closure_apply(c, d) : 0;
  /* reconstruction passes: a rejected cell with available face neighbours
   * takes their equal-weight mean (state and HoT, neighbour_mean); it becomes
   * available for the next pass */
  *n_rec = 0;
  uint8_t* nxt = (uint8_t*)malloc(n);
  for (int pass = 0; pass < c->cfg.passes; ++pass) {
    memcpy(nxt, avail, n);
    for (int64_t t = 0; t < n; ++t) {
      if (avail[t]) continue;
      if (!neighbour_mean(c, t, avail)) continue;
      nxt[t] = 1;
      c->cp_flag[t] = 2.0;
      (*n_rec)++;
    }
    memcpy(avail, nxt, n);
  }
  /* fill layers: rejected cells beyond the reconstruction layers still need a
   * state for the solve; they are filled the same way, layer by layer (flag 3,
   * not counted as reconstructed), until a layer fills nothing or after
   * ORC_FILL_LAYERS layers.  They are not recalibrated. */
  for (int layer = 0; layer < ORC_FILL_LAYERS; ++layer) {
    int64_t filled = 0;
    memcpy(nxt, avail, n);
    for (int64_t t = 0; t < n; ++t) {
      if (avail[t]) continue;
      if (!neighbour_mean(c, t, avail)) continue;
      nxt[t] = 1;
      c->cp_flag[t] = 3.0;
      filled++;
    }
    memcpy(avail, nxt, n);
    if (filled == 0) break;
  }
  /* a cell still without a state (no accepted cell connected to it within
   * the layers) starts the solve from the configuration's initial state
   * (density m n_init, velocity u_init, temperatures T_init: for an open
   * domain the free stream) with zero HoT; flag 0, not recalibrated */
  for (int64_t t = 0; t < n; ++t) {
    if (avail[t]) continue;
    double* h = c->cp_half + 6 * t;
    h[0] = 1.0;
    for (int i = 0; i < 3; ++i) h[1 + i] = c->cfg.u_init[i] / d->c0;
    h[4] = 1.0;
    h[5] = 1.0;
    memset(c->cp_hot + 12 * t, 0, 12 * sizeof(double));
  }
  free(nxt); free(avail); free(nbar);
}

/* S10 discretisation: steady synthetic equations (Eq. macro with the closure
 * sigma = sigma_NSF + HoT, q = q_NSF + HoT) by cell-centred finite volumes,
 * Rusanov inviscid flux with a low-Mach scaling of its velocity dissipation,
 * face-averaged stress and heat flux, diffuse walls as isothermal no-slip
 * walls and specular walls as slip walls (see the wall faces below), open
 * faces by the free stream.  The iteration is solve_synthetic below. */
static void prim_from_cons(const nd_t* d, const double* U, double* P) {
  const double rho = U[0];
  const double ux = U[1] / rho, uy = U[2] / rho, uz = U[3] / rho;
  const double er = d->dr > 0 ? U[5] / rho : 0.0;
  const double E = U[4] / rho;
  P[0] = rho; P[1] = ux; P[2] = uy; P[3] = uz;
  P[4] = (2.0 / 3.0) * (E - 0.5 * (ux * ux + uy * uy + uz * uz) - er);
  P[5] = d->dr > 0 ? 2.0 * er / d->dr : P[4];
}

static void cons_from_prim(const nd_t* d, const double* P, double* U) {
  const double rho = P[0], uu = P[1] * P[1] + P[2] * P[2] + P[3] * P[3];
  const double er = d->dr > 0 ? 0.5 * d->dr * P[5] : 0.0;
  U[0] = rho; U[1] = rho * P[1]; U[2] = rho * P[2]; U[3] = rho * P[3];
  U[4] = rho * (1.5 * P[4] + 0.5 * uu + er);
  U[5] = rho * er;
}

/* inviscid flux along unit normal N of primitive state P */
static void inv_flux(const double* P, const double* U, const double* N, double* F) {
  const double un = P[1] * N[0] + P[2] * N[1] + P[3] * N[2];
  const double p = P[0] * P[4];
  F[0] = U[0] * un;
  F[1] = U[1] * un + p * N[0];
  F[2] = U[2] * un + p * N[1];
  F[3] = U[3] * un + p * N[2];
  F[4] = (U[4] + p) * un;
  F[5] = U[5] * un;
}

/* Residual R(U) = -(1/V) sum_f F_f A_f (+ relaxation source, + src) of every
 * cell, and its pseudo-time step at CFL 1, dtl = V / sum_f A_f (lambda_f +
 * 2 nu A_f / V) with the face's largest inviscid wave speed lambda_f;
 * returns sum_c V_c |R_c|^2 over rho, rho u, rho E.  Work arrays: P [6n] primitives, G [15n] gradients, S [12n] total stress and
 * heat fluxes. */
static double residual(orc_ctx* c, const nd_t* d, const double* src, const double* U, double* R, double* dtl,
                       double* P, double* G, double* S) {
  const int64_t n = c->n_tets;
  const int nv = 6;
  const double L2 = d->L0 * d->L0, L3 = L2 * d->L0;
  for (int64_t t = 0; t < n; ++t) prim_from_cons(d, U + nv * t, P + 6 * t);
  gradients(c, d, P, G);
  for (int64_t t = 0; t < n; ++t) {
    double sig[6], qt[3], qr[3];
    nsf(d, P + 6 * t, G + 15 * t, sig, qt, qr);
    const double* H = c->cp_hot + 12 * t;
    for (int q = 0; q < 6; ++q) S[12 * t + q] = sig[q] + H[q];
    for (int q = 0; q < 3; ++q) {
      S[12 * t + 6 + q] = qt[q] + H[6 + q];
      S[12 * t + 9 + q] = qr[q] + H[9 + q];
    }
  }
  double rsum = 0.0;
  for (int64_t t = 0; t < n; ++t) {
    const double* Pc = P + 6 * t;
    const double* Uc = U + nv * t;
    const double V = c->vol[t] / L3;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    double lam_sum = 0.0;
    const double cc = sqrt(d->gam * Pc[4]);
    const double nu = 2.5 * mu_nd(d, Pc[4]) / Pc[0];
    for (int f = 0; f < 4; ++f) {
      const double* N = c->pn + 12 * t + 3 * f;
      const double A = c->parea[4 * t + f] / L2;
      const int32_t nb = c->nbr[4 * t + f];
      double F[6];
      if (nb >= 0 || c->bcs[c->bf[-1 - nb].bc].kind >= 2) {
        double Pn[6], Un[6];
        if (nb >= 0) {
          memcpy(Pn, P + 6 * (int64_t)nb, sizeof Pn);
          memcpy(Un, U + nv * (int64_t)nb, sizeof Un);
        } else {
          const orc_bc* b = c->bcs + c->bf[-1 - nb].bc;
          Pn[0] = b->kind == 2 ? b->n * c->cfg.mass / d->rho0 : Pc[0];
          Pn[1] = b->U[0] / d->c0; Pn[2] = b->U[1] / d->c0; Pn[3] = b->U[2] / d->c0;
          Pn[4] = b->T / d->T0; Pn[5] = Pn[4];
          if (b->kind == 3) memcpy(Pn, Pc, sizeof Pn);
          cons_from_prim(d, Pn, Un);
        }
        double FL[6], FR[6];
        inv_flux(Pc, Uc, N, FL);
        inv_flux(Pn, Un, N, FR);
        const double unl = Pc[1] * N[0] + Pc[2] * N[1] + Pc[3] * N[2];
        const double unr = Pn[1] * N[0] + Pn[2] * N[1] + Pn[3] * N[2];
        const double cl = sqrt(d->gam * Pc[4]), cr = sqrt(d->gam * (Pn[4] > 0 ? Pn[4] : 1e-12));
        const double lm = fmax(fabs(unl) + cl, fabs(unr) + cr);
        if (nb >= 0) {
          /* interior face: the dissipation acts on states whose velocity
           * jump is scaled by z = min(1, max(M_L, M_R)) (low-Mach correction
           * of Thornber et al. 2008) and whose density jump keeps its
           * acoustic part dp / c^2 and scales its entropy part
           * drho - dp / c^2 by z (c^2 = gamma T of the face mean), with
           * the pressures unchanged: at low Mach the dissipation of shear
           * and entropy waves scales with the flow speed instead of the
           * sound speed */
          const double ml = sqrt(Pc[1] * Pc[1] + Pc[2] * Pc[2] + Pc[3] * Pc[3]) / cl;
          const double mr = sqrt(Pn[1] * Pn[1] + Pn[2] * Pn[2] + Pn[3] * Pn[3]) / cr;
          const double z = fmin(1.0, fmax(ml, mr));
          double PL[6], PR[6], UL[6], UR[6];
          memcpy(PL, Pc, sizeof PL);
          memcpy(PR, Pn, sizeof PR);
          for (int i = 1; i <= 3; ++i) {
            const double m = 0.5 * (Pc[i] + Pn[i]), h = 0.5 * z * (Pc[i] - Pn[i]);
            PL[i] = m + h;
            PR[i] = m - h;
          }
          const double pl = Pc[0] * Pc[4], pr = Pn[0] * Pn[4];
          const double c2 = d->gam * 0.5 * (Pc[4] + Pn[4]);
          const double dpc = (pl - pr) / c2;
          const double drho = dpc + z * ((Pc[0] - Pn[0]) - dpc);
          const double rm = 0.5 * (Pc[0] + Pn[0]);
          PL[0] = rm + 0.5 * drho;
          PR[0] = rm - 0.5 * drho;
          PL[4] = pl / PL[0];
          PR[4] = pr / PR[0];
          cons_from_prim(d, PL, UL);
          cons_from_prim(d, PR, UR);
          for (int q = 0; q < 6; ++q) F[q] = 0.5 * (FL[q] + FR[q]) - 0.5 * lm * (UR[q] - UL[q]);
        } else {
          for (int q = 0; q < 6; ++q) F[q] = 0.5 * (FL[q] + FR[q]) - 0.5 * lm * (Un[q] - Uc[q]);
        }
        if (nb >= 0) {
          const double* Sc = S + 12 * t;
          const double* Sn = S + 12 * (int64_t)nb;
          double sf[6], qtf[3], qrf[3], uf[3];
          for (int q = 0; q < 6; ++q) sf[q] = 0.5 * (Sc[q] + Sn[q]);
          for (int q = 0; q < 3; ++q) {
            qtf[q] = 0.5 * (Sc[6 + q] + Sn[6 + q]);
            qrf[q] = 0.5 * (Sc[9 + q] + Sn[9 + q]);
            uf[q] = 0.5 * (Pc[1 + q] + Pn[1 + q]);
          }
          /* sigma . n with sigma = [[xx,xy,xz],[xy,yy,yz],[xz,yz,zz]] */
          const double sn0 = sf[0] * N[0] + sf[3] * N[1] + sf[4] * N[2];
          const double sn1 = sf[3] * N[0] + sf[1] * N[1] + sf[5] * N[2];
          const double sn2 = sf[4] * N[0] + sf[5] * N[1] + sf[2] * N[2];
          F[1] += sn0; F[2] += sn1; F[3] += sn2;
          F[4] += sn0 * uf[0] + sn1 * uf[1] + sn2 * uf[2] + (qtf[0] + qrf[0]) * N[0] + (qtf[1] + qrf[1]) * N[1] +
                  (qtf[2] + qrf[2]) * N[2];
          F[5] += qrf[0] * N[0] + qrf[1] * N[1] + qrf[2] * N[2];
        }
        lam_sum += A * (lm + 2.0 * nu * A / V);
      } else {
        /* wall: no mass flux.  A diffuse wall closes the equations as an
         * isothermal no-slip wall: the cell's pressure and total stress
         * (NSF from gradients that take the wall velocity and temperature
         * at the face, plus the cell's HoT) plus the numerical friction
         * below, the work of both at the wall velocity and the cell's heat
         * fluxes.  A specular wall carries the cell's pressure only. */
        const int32_t ib = -1 - nb;
        const orc_bc* bw = c->bcs + c->bf[ib].bc;
        const double p = Pc[0] * Pc[4];
        F[0] = 0.0;
        if (bw->kind == 0) {
          const double* Sc = S + 12 * t;
          const double Uw[3] = {bw->U[0] / d->c0, bw->U[1] / d->c0, bw->U[2] / d->c0};
          const double sn0 = Sc[0] * N[0] + Sc[3] * N[1] + Sc[4] * N[2];
          const double sn1 = Sc[3] * N[0] + Sc[1] * N[1] + Sc[5] * N[2];
          const double sn2 = Sc[4] * N[0] + Sc[5] * N[1] + Sc[2] * N[2];
          /* the interior faces' dissipation against the mirrored ghost
           * state (velocity 2 U_w - u): a friction lambda z rho (U_w - u),
           * lambda = |u.n| + c, z = min(1, max(|u|/c, |U_w|/c)), whose work
           * is done at the wall velocity */
          const double z = fmin(1.0, fmax(sqrt(Pc[1] * Pc[1] + Pc[2] * Pc[2] + Pc[3] * Pc[3]) / cc,
                                          sqrt(Uw[0] * Uw[0] + Uw[1] * Uw[1] + Uw[2] * Uw[2]) / cc));
          const double kw = (fabs(Pc[1] * N[0] + Pc[2] * N[1] + Pc[3] * N[2]) + cc) * z * Pc[0];
          double fw[3];
          for (int i = 0; i < 3; ++i) fw[i] = -kw * (Uw[i] - Pc[1 + i]);
          F[1] = p * N[0] + sn0 + fw[0];
          F[2] = p * N[1] + sn1 + fw[1];
          F[3] = p * N[2] + sn2 + fw[2];
          F[4] = (sn0 + fw[0]) * Uw[0] + (sn1 + fw[1]) * Uw[1] + (sn2 + fw[2]) * Uw[2] + (Sc[6] + Sc[9]) * N[0] +
                 (Sc[7] + Sc[10]) * N[1] + (Sc[8] + Sc[11]) * N[2];
          F[5] = Sc[9] * N[0] + Sc[10] * N[1] + Sc[11] * N[2];
        } else {
          for (int i = 0; i < 3; ++i) F[1 + i] = p * N[i];
          F[4] = 0.0;
          F[5] = 0.0;
        }
        /* wave speed of the wall face: |u.n| + c, as for the interior faces */
        lam_sum += A * (fabs(Pc[1] * N[0] + Pc[2] * N[1] + Pc[3] * N[2]) + cc + 2.0 * nu * A / V);
      }
      for (int q = 0; q < 6; ++q) acc[q] += F[q] * A;
    }
    double* Rc = R + nv * t;
    for (int q = 0; q < 6; ++q) Rc[q] = -acc[q] / V;
    if (d->dr > 0) {
      /* rotational relaxation source (Eq. macro, last line) */
      const double T = (3.0 * Pc[4] + d->dr * Pc[5]) / (3.0 + d->dr);
      const double tau = mu_nd(d, Pc[4]) / (Pc[0] * Pc[4]);
      Rc[5] += 0.5 * d->dr * Pc[0] * (T - Pc[5]) / (d->Zr * tau);
    } else {
      Rc[5] = 0.0;
    }
    /* a given volume source (the manufactured-solution pin only) */
    if (src)
      for (int q = 0; q < 6; ++q) Rc[q] += src[6 * t + q];
    dtl[t] = V / lam_sum;
    for (int q = 0; q < 5; ++q) rsum += V * Rc[q] * Rc[q];
  }
  return rsum;
}

/* Inner product of two state vectors [n][6] weighted by the cell volumes
 * (nondimensional), summed cell by cell in index order. */
static double wdot(const double* a, const double* b, const double* w, int64_t n) {
  double s = 0.0;
  for (int64_t t = 0; t < n; ++t) {
    double r = 0.0;
    for (int q = 0; q < 6; ++q) r += a[6 * t + q] * b[6 * t + q];
    s += w[t] * r;
  }
  return s;
}

/* The coefficients gamma minimising |f - dF gamma| (volume-weighted norm)
 * over the k held columns, in age order (oldest first), from the Gram
 * matrix H of the columns and b_i = <dF_i, f> (both held by ring slot):
 * normal equations of the columns scaled to unit norm, with 1e-10 added to
 * the diagonal, by Cholesky.  Returns 0 if the factorisation fails (then no
 * column is used). */
static int aa_coefficients(const double (*Hs)[ORC_AA_MAX], const double* bs, const int* slot, int k, double* gam) {
  double H[ORC_AA_MAX][ORC_AA_MAX], b[ORC_AA_MAX], sc[ORC_AA_MAX], y[ORC_AA_MAX];
  for (int i = 0; i < k; ++i) {
    for (int j = 0; j < k; ++j) H[i][j] = Hs[slot[i]][slot[j]];
    b[i] = bs[slot[i]];
  }
  for (int i = 0; i < k; ++i) sc[i] = H[i][i] > 0 ? 1.0 / sqrt(H[i][i]) : 0.0;
  for (int i = 0; i < k; ++i) {
    for (int j = 0; j < k; ++j) H[i][j] *= sc[i] * sc[j];
    H[i][i] += 1e-10;
    b[i] *= sc[i];
  }
  for (int j = 0; j < k; ++j) {
    double d = H[j][j];
    for (int q = 0; q < j; ++q) d -= H[j][q] * H[j][q];
    if (!(d > 0)) return 0;
    H[j][j] = sqrt(d);
    for (int i = j + 1; i < k; ++i) {
      double e = H[i][j];
      for (int q = 0; q < j; ++q) e -= H[i][q] * H[j][q];
      H[i][j] = e / H[j][j];
    }
  }
  for (int i = 0; i < k; ++i) {
    double e = b[i];
    for (int q = 0; q < i; ++q) e -= H[i][q] * y[q];
    y[i] = e / H[i][i];
  }
  for (int i = k - 1; i >= 0; --i) {
    double e = y[i];
    for (int q = i + 1; q < k; ++q) e -= H[q][i] * gam[q];
    gam[i] = e / H[i][i];
  }
  for (int i = 0; i < k; ++i) gam[i] *= sc[i];
  return 1;
}

/* S10: the steady synthetic equations (Eq. macro with the closure of Eq.
 * synthetic_closure) solved by pseudo-time iteration.  The base step is the
 * forward-Euler step of each cell's own pseudo-time step (CFL cfg.cfl of its
 * inviscid and viscous wave speeds), g(U) = U + cfl dtl R(U), the step of a
 * cell halved while it would leave a non-positive density or temperature
 * there (at most 11 times; a cell still not positive keeps its state: at a
 * fixed point no halving occurs); without open boundaries it is followed by a
 * scaling of every conserved variable that
 * restores the initial total mass (local steps do not conserve it, and the
 * steady equations of a closed domain leave it free).  Anderson acceleration
 * of depth m = cfg.aa_m (Walker & Ni, SIAM J. Numer. Anal. 49, 2011) combines
 * the last m steps: U <- g(U_k) - dG gamma, gamma minimising
 * |f_k - dF gamma| with f = g(U) - U and dF, dG the differences of
 * consecutive f and g(U).  The Gram matrix H_ij = <dF_i, dF_j> gains one
 * row per iteration (the new column against every held one), and
 * b_i = <dF_i, f_k> follows from f_k = f_{k-1} + dF_new as b_i + H_i,new,
 * except for the new column's, which is computed.  A combined state with a
 * non-positive density or temperature in some cell is replaced by g(U_k),
 * and the history is cleared.  A non-finite residual, or one above 100 times
 * the best so far, sends the iteration back to the best iterate with half
 * the CFL number (at most six times) and no history.  Stops after N_m
 * iterations or when the residual norm falls to eps_m times its first
 * value; the result is the last iterate, or the best one if the last is
 * worse. */
static int solve_synthetic(orc_ctx* c, const nd_t* d, const double* src, int* iters, double* res_out) {
  const int64_t n = c->n_tets;
  const int nv = 6;
  const int64_t len = nv * n;
  const int m = c->cfg.aa_m < 0 ? 0 : c->cfg.aa_m > ORC_AA_MAX ? ORC_AA_MAX : c->cfg.aa_m;
  double cfl = c->cfg.cfl > 0 ? c->cfg.cfl : 1.5;
  const double cfl_min = cfl / 64.0;
  double* U = (double*)malloc(sizeof(double) * len);
  double* Ub = (double*)malloc(sizeof(double) * len); /* the best iterate so far */
  double* P = (double*)calloc(6 * n, sizeof(double));
  double* R = (double*)malloc(sizeof(double) * len);
  double* G = (double*)malloc(sizeof(double) * 15 * n);
  double* S = (double*)malloc(sizeof(double) * 12 * n);
  double* dtl = (double*)malloc(sizeof(double) * n);
  double* w = (double*)malloc(sizeof(double) * n);
  double* Gx = (double*)malloc(sizeof(double) * len);
  double* f = (double*)malloc(sizeof(double) * len);
  double* fp = (double*)malloc(sizeof(double) * len);
  double* Gp = (double*)malloc(sizeof(double) * len);
  double* dF = (double*)malloc(sizeof(double) * len * (m > 0 ? m : 1));
  double* dG = (double*)malloc(sizeof(double) * len * (m > 0 ? m : 1));
  const double L3 = d->L0 * d->L0 * d->L0;
  int closed = 1;
  for (int32_t i = 0; i < c->n_bf; ++i)
    if (c->bcs[c->bf[i].bc].kind >= 2) closed = 0;
  double M0 = 0.0;
  for (int64_t t = 0; t < n; ++t) {
    cons_from_prim(d, c->cp_half + 6 * t, U + nv * t);
    w[t] = c->vol[t] / L3;
    M0 += w[t] * U[nv * t];
  }
  double res0 = 0.0, res = 0.0, resb = 0.0;
  double Hs[ORC_AA_MAX][ORC_AA_MAX], bs[ORC_AA_MAX];
  int it = 0, nh = 0, head = 0, fresh = 1; /* fresh: no previous f to difference with */
  for (it = 0; it < c->cfg.N_m; ++it) {
    res = sqrt(residual(c, d, src, U, R, dtl, P, G, S));
    if (it == 0) {
      res0 = res > 0 ? res : 1.0;
      resb = res;
      memcpy(Ub, U, sizeof(double) * len);
    }
    if (res <= c->cfg.eps_m * res0) break;
    /* divergence (a non-finite residual or one 100 times the best): back to
     * the best iterate with half the CFL number (down to 1/64 of the
     * configured one) and no history; the next iteration starts there */
    if (!(res <= 100.0 * resb)) {
      if (cfl <= cfl_min) break;
      memcpy(U, Ub, sizeof(double) * len);
      cfl = 0.5 * cfl;
      nh = 0;
      fresh = 1;
      continue;
    }
    if (res < resb) {
      resb = res;
      memcpy(Ub, U, sizeof(double) * len);
    }
    /* base step, each cell's own step halved until its state stays positive
     * (at most 11 times, then the cell keeps its state) */
    for (int64_t t = 0; t < n; ++t) {
      double dt = cfl * dtl[t];
      for (int h = 0; h < 12; ++h) {
        double* G = Gx + nv * t;
        for (int q = 0; q < nv; ++q) G[q] = U[nv * t + q] + dt * R[nv * t + q];
        /* rho > 0 and T_t > 0, the latter as rho (rho E) - |rho u|^2 / 2 - rho (rho e_r) > 0 */
        if (G[0] > 0 && G[0] * G[4] - 0.5 * (G[1] * G[1] + G[2] * G[2] + G[3] * G[3]) - G[0] * G[5] > 0) break;
        dt = h < 10 ? 0.5 * dt : 0.0;
      }
    }
    if (closed) {
      double Mx = 0.0;
      for (int64_t t = 0; t < n; ++t) Mx += w[t] * Gx[nv * t];
      const double sc = M0 / Mx;
      for (int64_t i = 0; i < len; ++i) Gx[i] *= sc;
    }
    if (m == 0) {
      memcpy(U, Gx, sizeof(double) * len);
      continue;
    }
    /* acceleration */
    for (int64_t i = 0; i < len; ++i) f[i] = Gx[i] - U[i];
    int slot[ORC_AA_MAX];
    double gam[ORC_AA_MAX];
    if (!fresh) {
      const int s0 = head;
      double* a = dF + len * s0;
      double* b = dG + len * s0;
      for (int64_t i = 0; i < len; ++i) {
        a[i] = f[i] - fp[i];
        b[i] = Gx[i] - Gp[i];
      }
      head = (head + 1) % m;
      if (nh < m) nh++;
      for (int i = 0; i < nh; ++i) slot[i] = ((head - nh + i) % m + m) % m;
      for (int i = 0; i < nh; ++i) {
        const double h = wdot(dF + len * slot[i], a, w, n);
        Hs[slot[i]][s0] = Hs[s0][slot[i]] = h;
        if (slot[i] != s0) bs[slot[i]] += h;
      }
      bs[s0] = wdot(a, f, w, n);
    }
    fresh = 0;
    memcpy(fp, f, sizeof(double) * len);
    memcpy(Gp, Gx, sizeof(double) * len);
    for (int i = 0; i < nh; ++i) slot[i] = ((head - nh + i) % m + m) % m;
    const int k = nh > 0 && aa_coefficients(Hs, bs, slot, nh, gam) ? nh : 0;
    int pos = 1;
    for (int64_t t = 0; t < n; ++t) {
      for (int q = 0; q < nv; ++q) {
        double x = Gx[nv * t + q];
        for (int j = 0; j < k; ++j) x -= gam[j] * dG[len * slot[j] + nv * t + q];
        U[nv * t + q] = x;
      }
      double Pp[6];
      prim_from_cons(d, U + nv * t, Pp);
      if (!(Pp[0] > 0 && Pp[4] > 0)) pos = 0;
    }
    if (!pos) {
      memcpy(U, Gx, sizeof(double) * len);
      nh = 0;
    }
  }
  /* the result: the last iterate, or the best one if the last is worse (a
   * stop at N_m after a rise of the residual, or a divergence) */
  if (!(res <= resb)) {
    memcpy(U, Ub, sizeof(double) * len);
    res = resb;
  }
  int ok = isfinite(res);
  for (int64_t t = 0; t < n && ok; ++t) {
    prim_from_cons(d, U + nv * t, c->cp_new + 6 * t);
    ok = c->cp_new[6 * t] > 0 && c->cp_new[6 * t + 4] > 0;
  }
  *iters = it;
  *res_out = res / res0;
  free(U); free(Ub); free(P); free(R); free(G); free(S); free(dtl); free(w); free(Gx); free(f); free(fp); free(Gp);
  free(dF); free(dG);
  return ok ? 0 : -5;
}

/* S11: recalibrate the particles of accepted cells to M^{k+1}:
 * v' = u_a + (v - u_b) sqrt(T_a / T_b), I' = I T_r,a / T_r,b (ratios clamped
 * to [1/4, 4]); number ratio r = rho_a / rho_N clamped to [1/2, 2]: delete
 * with probability 1 - r, or clone with probability r - 1 (the clone at a
 * uniform point of the cell with the recalibrated velocity).  b = the cell's
 * own sampled state (moving average), a = the solved state, rho_N = m F_N N_c
 * / V the density of the N_c particles the cell holds now, so that the
 * expected count after the adjustment is rho_a V / (m F_N): the particles are
 * resampled to M^{k+1} and the mass the solve conserves is the particles'. */
static void recalibrate(orc_ctx* c, const nd_t* d, int64_t* n_clone, int64_t* n_del) {
  const int64_t n = c->n_tets, N = c->N;
  *n_clone = 0;
  *n_del = 0;
  int64_t cap_moved = N + N / 4 + 1024;
  uint8_t* moved = (uint8_t*)calloc((size_t)cap_moved, 1);
  const uint32_t sub = (uint32_t)c->n_couple;
  for (int64_t t = 0; t < n; ++t) {
    if (c->cp_flag[t] != 1.0) continue;
    const double* b = c->cp_own + 6 * t;
    const double* a = c->cp_new + 6 * t;
    double rt = a[4] / b[4];
    rt = rt < 0.25 ? 0.25 : rt > 4.0 ? 4.0 : rt;
    double rr = d->dr > 0 ? a[5] / b[5] : 1.0;
    rr = rr < 0.25 ? 0.25 : rr > 4.0 ? 4.0 : rr;
    const int64_t Nc = c->cstart[t + 1] - c->cstart[t];
    const double rho_N = c->cfg.mass * c->cfg.F_N * (double)Nc / c->vol[t] / d->rho0;
    double rn = Nc > 0 ? a[0] / rho_N : 1.0;
    rn = rn < 0.5 ? 0.5 : rn > 2.0 ? 2.0 : rn;
    const vreal sc = (vreal)sqrt(rt), fr = (vreal)rr;
    vreal ua[3], ub[3];
    for (int i = 0; i < 3; ++i) {
      ua[i] = (vreal)(a[1 + i] * d->c0);
      ub[i] = (vreal)(b[1 + i] * d->c0);
    }
    for (int64_t p = c->cstart[t]; p < c->cstart[t + 1]; ++p) {
      vreal* v = c->v + 3 * p;
      for (int i = 0; i < 3; ++i) v[i] = ua[i] + (v[i] - ub[i]) * sc;
      c->Ir[p] = c->Ir[p] * fr;
      uint32_t w[4];
      rng4(c, RP_RECAL, (uint32_t)p, sub, 0, 0, w);
      const double R = u01d(w[0], w[1]);
      if (rn < 1.0) {
        if (R < 1.0 - rn) {
          c->cell[p] = -1;
          (*n_del)++;
        }
      } else if (rn > 1.0 && R < rn - 1.0) {
        const int64_t q = c->N;
        ensure_cap(c, q + 1);
        if (q + 1 > cap_moved) {
          cap_moved = 2 * (q + 1);
          moved = (uint8_t*)realloc(moved, (size_t)cap_moved);
        }
        uint32_t w2[4];
        rng4(c, RP_RECAL, (uint32_t)p, sub, 0, 1, w);
        rng4(c, RP_RECAL, (uint32_t)p, sub, 0, 2, w2);
        double s = u01d(w[0], w[1]), tt = u01d(w[2], w[3]), u = u01d(w2[0], w2[1]);
        if (s + tt > 1.0) { s = 1.0 - s; tt = 1.0 - tt; }
        if (tt + u > 1.0) {
          double tmp = u; u = 1.0 - s - tt; tt = 1.0 - tmp;
        } else if (s + tt + u > 1.0) {
          double tmp = u; u = s + tt + u - 1.0; s = 1.0 - tt - tmp;
        }
        const double* A = c->nodes + 3 * c->tets[4 * t + 0];
        const double* B = c->nodes + 3 * c->tets[4 * t + 1];
        const double* C = c->nodes + 3 * c->tets[4 * t + 2];
        const double* D = c->nodes + 3 * c->tets[4 * t + 3];
        for (int i = 0; i < 3; ++i)
          c->x[3 * q + i] = A[i] + s * (B[i] - A[i]) + tt * (C[i] - A[i]) + u * (D[i] - A[i]);
        memcpy(c->v + 3 * q, c->v + 3 * p, 3 * sizeof(vreal));
        c->Ir[q] = c->Ir[p];
        c->cell[q] = (int32_t)t;
        moved[q] = 1;
        c->N = q + 1;
        (*n_clone)++;
      }
    }
  }
  sort_particles(c, moved);
  free(moved);
}

int orc_couple(orc_ctx* c, orc_couple_report* rep) {
  if (!c->vol) return fail(c, -7, "mesh not loaded");
  const int64_t n = c->n_tets;
  if (!c->cp_half) {
    c->cp_half = (double*)calloc(6 * n, sizeof(double));
    c->cp_hot = (double*)calloc(12 * n, sizeof(double));
    c->cp_new = (double*)calloc(6 * n, sizeof(double));
    c->cp_own = (double*)calloc(6 * n, sizeof(double));
    c->cp_flag = (double*)calloc(n, sizeof(double));
  }
  const nd_t d = nondim(c);
  memset(rep, 0, sizeof *rep);
  int64_t n_learned = 0;
  extract_hot(c, &d, &rep->n_rejected, &rep->n_reconstructed, &n_learned);
  rep->n_learned = (int32_t)n_learned;
  int rc = solve_synthetic(c, &d, NULL, &rep->iters, &rep->residual);
  /* the k-th coupling (k = 0, 1, ...) keys its random stream with sub = k */
  if (rc == 0) recalibrate(c, &d, &rep->n_cloned, &rep->n_deleted);
  c->n_couple++;
  memset(c->bflux, 0, sizeof(double) * 5 * (c->n_bf > 0 ? c->n_bf : 1));
  c->flux_steps = 0;
  return rc == 0 ? 0 : fail(c, -5, "synthetic solve failed (non-finite or non-positive state)");
}

/* Harness exports for the pins of the synthetic equations (Sec. 2.2): the
 * least-squares gradients, the NSF relations and the solve itself, each run
 * on a state the caller gives (nondimensional, rows per cell). */
int orc_gradients(orc_ctx* c, const double* prim, double* grad) {
  if (!c->vol) return fail(c, -7, "mesh not loaded");
  const nd_t d = nondim(c);
  gradients(c, &d, prim, grad);
  return 0;
}

int orc_nsf(orc_ctx* c, const double* prim, const double* grad, double* out) {
  if (!c->vol) return fail(c, -7, "mesh not loaded");
  const nd_t d = nondim(c);
  for (int64_t t = 0; t < c->n_tets; ++t) nsf(&d, prim + 6 * t, grad + 15 * t, out + 12 * t, out + 12 * t + 6,
                                               out + 12 * t + 9);
  return 0;
}

int orc_synthetic_residual(orc_ctx* c, const double* prim, const double* hot, const double* src, double* R,
                           double* dtl) {
  if (!c->vol) return fail(c, -7, "mesh not loaded");
  const int64_t n = c->n_tets;
  if (!c->cp_hot) c->cp_hot = (double*)calloc(12 * n, sizeof(double));
  memcpy(c->cp_hot, hot, sizeof(double) * 12 * n);
  const nd_t d = nondim(c);
  double* U = (double*)malloc(sizeof(double) * 6 * n);
  double* P = (double*)calloc(6 * n, sizeof(double));
  double* G = (double*)malloc(sizeof(double) * 15 * n);
  double* S = (double*)malloc(sizeof(double) * 12 * n);
  for (int64_t t = 0; t < n; ++t) cons_from_prim(&d, prim + 6 * t, U + 6 * t);
  residual(c, &d, src, U, R, dtl, P, G, S);
  free(U); free(P); free(G); free(S);
  return 0;
}

int orc_synthetic_solve(orc_ctx* c, const double* half, const double* hot, const double* src, double* out,
                        int32_t* iters, double* res) {
  if (!c->vol) return fail(c, -7, "mesh not loaded");
  const int64_t n = c->n_tets;
  if (!c->cp_half) {
    c->cp_half = (double*)calloc(6 * n, sizeof(double));
    c->cp_hot = (double*)calloc(12 * n, sizeof(double));
    c->cp_new = (double*)calloc(6 * n, sizeof(double));
    c->cp_own = (double*)calloc(6 * n, sizeof(double));
    c->cp_flag = (double*)calloc(n, sizeof(double));
  }
  memcpy(c->cp_half, half, sizeof(double) * 6 * n);
  memcpy(c->cp_hot, hot, sizeof(double) * 12 * n);
  const nd_t d = nondim(c);
  int it = 0;
  const int rc = solve_synthetic(c, &d, src, &it, res);
  *iters = it;
  memcpy(out, c->cp_new, sizeof(double) * 6 * n);
  return rc == 0 ? 0 : fail(c, -5, "synthetic solve failed (non-finite or non-positive state)");
}

int orc_read_couple(orc_ctx* c, int32_t which, double* out, int64_t cap) {
  const int64_t n = c->n_tets;
  if (which < 0 || which > 5) return fail(c, -1, "bad selector");
  const double* src = which == 0 ? c->cp_half : which == 1 ? c->cp_hot : which == 2 ? c->cp_new
                    : which == 3 ? c->cp_flag : which == 4 ? c->cp_own : c->acc_w;
  const int64_t k = which == 1 ? 12 : which == 3 || which == 5 ? 1 : 6;
  if (!src) return fail(c, -7, "no coupling done");
  if (cap < k * n) return fail(c, -3, "buffer too small");
  memcpy(out, src, sizeof(double) * k * n);
  return 0;
}

int orc_write_moments(orc_ctx* c, int32_t which, const double* in) {
  const int64_t n = c->n_tets;
  double* dst = which == ORC_PHI_INST ? c->phi_inst : which == ORC_PHI_EWMA ? c->phi_ewma
              : which == ORC_PHI_WINDOW ? c->phi_win : c->phi_cum;
  memcpy(dst, in, sizeof(double) * NPHI_MAX * n);
  if (which == ORC_PHI_EWMA && c->n_ewma == 0) c->n_ewma = 1;
  return 0;
}

int orc_write_wall_flux(orc_ctx* c, const double* in, int64_t steps) {
  memcpy(c->bflux, in, sizeof(double) * 5 * c->n_bf);
  c->flux_steps = steps;
  return 0;
}

/* ========================================================================= */
/* S12/S13: learned per-cell closure (not in the paper): an MLP             */
/* 13 -> 64 -> 64 -> 64 -> 8 with GELU, BF16 weights and activations,       */
/* accumulation in FP64 here (the reference of the FP32-accumulating        */
/* kernels).  Parameters, FP32 master copy, layout [out][in] per layer:     */
/* W1[64][13] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[8][64] b4[8].   */
/* ========================================================================= */
#define MLP_NIN 13
#define MLP_NH 64
#define MLP_NOUT 8
#define MLP_NPARAM (MLP_NH * MLP_NIN + MLP_NH + 2 * (MLP_NH * MLP_NH + MLP_NH) + MLP_NOUT * MLP_NH + MLP_NOUT)

int32_t orc_mlp_nparam(void) { return MLP_NPARAM; }

/* FP32 -> BF16 -> FP32, round to nearest even */
double orc_bf16(double x) {
  float f = (float)x;
  uint32_t b;
  memcpy(&b, &f, 4);
  if ((b & 0x7f800000u) == 0x7f800000u) return f; /* inf / nan unchanged */
  b = (b + 0x7fffu + ((b >> 16) & 1u)) & 0xffff0000u;
  memcpy(&f, &b, 4);
  return f;
}

static double gelu(double z) { return 0.5 * z * (1.0 + erf(z / sqrt(2.0))); }
static double gelu_d(double z) { return 0.5 * (1.0 + erf(z / sqrt(2.0))) + z * exp(-0.5 * z * z) / sqrt(2.0 * M_PI); }

typedef struct {
  const float *W[4], *b[4];
  int nin[4], nout[4];
} mlp_view;

static mlp_view mlp_layout(const float* p) {
  mlp_view v;
  const int ni[4] = {MLP_NIN, MLP_NH, MLP_NH, MLP_NH}, no[4] = {MLP_NH, MLP_NH, MLP_NH, MLP_NOUT};
  const float* q = p;
  for (int l = 0; l < 4; ++l) {
    v.W[l] = q;
    q += ni[l] * no[l];
    v.b[l] = q;
    q += no[l];
    v.nin[l] = ni[l];
    v.nout[l] = no[l];
  }
  return v;
}

/* forward of one row; a[l] are the layer inputs (BF16-rounded when bf16 != 0),
 * z[l] the pre-activations; returns outputs y[8] */
static void mlp_row(const mlp_view* v, const float* x, int bf16, double a[4][MLP_NH], double z[4][MLP_NH], double* y) {
  for (int k = 0; k < MLP_NIN; ++k) a[0][k] = bf16 ? orc_bf16(x[k]) : x[k];
  for (int l = 0; l < 4; ++l) {
    for (int j = 0; j < v->nout[l]; ++j) {
      double s = 0.0;
      for (int k = 0; k < v->nin[l]; ++k) {
        double w = v->W[l][j * v->nin[l] + k];
        if (bf16) w = orc_bf16(w);
        s += w * a[l][k];
      }
      s += v->b[l][j];
      z[l][j] = s;
      if (l < 3) a[l + 1][j] = bf16 ? orc_bf16(gelu(s)) : gelu(s);
      else y[j] = s;
    }
  }
}

int orc_mlp_forward(const float* params, const float* X, int64_t n, int32_t bf16, double* Y) {
  mlp_view v = mlp_layout(params);
  double a[4][MLP_NH], z[4][MLP_NH];
  for (int64_t r = 0; r < n; ++r) mlp_row(&v, X + MLP_NIN * r, bf16, a, z, Y + MLP_NOUT * r);
  return 0;
}

/* mean-square loss L = 1/(8n) sum (y - t)^2 and its gradient with respect to
 * every parameter (backpropagation through the same computation; the BF16
 * roundings are passed straight through) */
double orc_mlp_grad(const float* params, const float* X, const float* T, int64_t n, int32_t bf16, double* grad) {
  mlp_view v = mlp_layout(params);
  memset(grad, 0, sizeof(double) * MLP_NPARAM);
  double* gW[4];
  double* gb[4];
  {
    double* q = grad;
    for (int l = 0; l < 4; ++l) {
      gW[l] = q;
      q += v.nin[l] * v.nout[l];
      gb[l] = q;
      q += v.nout[l];
    }
  }
  double loss = 0.0;
  double a[4][MLP_NH], z[4][MLP_NH], y[MLP_NOUT], d[MLP_NH], dn[MLP_NH];
  for (int64_t r = 0; r < n; ++r) {
    mlp_row(&v, X + MLP_NIN * r, bf16, a, z, y);
    for (int j = 0; j < MLP_NOUT; ++j) {
      const double e = y[j] - T[MLP_NOUT * r + j];
      loss += e * e;
      d[j] = 2.0 * e / (double)(MLP_NOUT * n);
    }
    for (int l = 3; l >= 0; --l) {
      for (int j = 0; j < v.nout[l]; ++j) {
        gb[l][j] += d[j];
        for (int k = 0; k < v.nin[l]; ++k) gW[l][j * v.nin[l] + k] += d[j] * a[l][k];
      }
      if (l == 0) break;
      for (int k = 0; k < v.nin[l]; ++k) {
        double s = 0.0;
        for (int j = 0; j < v.nout[l]; ++j) {
          double w = v.W[l][j * v.nin[l] + k];
          if (bf16) w = orc_bf16(w);
          s += w * d[j];
        }
        dn[k] = s * gelu_d(z[l - 1][k]);
      }
      memcpy(d, dn, sizeof(double) * v.nin[l]);
    }
  }
  return loss / (double)(MLP_NOUT * n);
}

/* Adam (Kingma and Ba 2015) on the FP32 master parameters, step t >= 1 */
void orc_adam(float* params, double* m, double* vv, const double* g, int64_t t, double lr, double b1, double b2,
              double eps) {
  const double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
  for (int i = 0; i < MLP_NPARAM; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    vv[i] = b2 * vv[i] + (1.0 - b2) * g[i] * g[i];
    params[i] = (float)(params[i] - lr * (m[i] / c1) / (sqrt(vv[i] / c2) + eps));
  }
}

/* He-normal initialisation from the MLP_INIT random stream (Box-Muller free:
 * polar Gaussian pairs), biases zero */
void orc_mlp_init(float* params, uint64_t seed) {
  orc_ctx tmp;
  memset(&tmp, 0, sizeof tmp);
  tmp.cfg.seed = seed;
  mlp_view v = mlp_layout(params);
  int idx = 0;
  for (int l = 0; l < 4; ++l) {
    const float sd = (float)sqrt(2.0 / v.nin[l]);
    float* W = (float*)v.W[l];
    float* b = (float*)v.b[l];
    for (int i = 0; i < v.nin[l] * v.nout[l]; i += 2, idx += 2) {
      vreal g1, g2;
      gauss2(&tmp, 9, (uint32_t)idx, 0, 0, 0, &g1, &g2);
      W[i] = (float)(sd * g1);
      if (i + 1 < v.nin[l] * v.nout[l]) W[i + 1] = (float)(sd * g2);
    }
    for (int j = 0; j < v.nout[l]; ++j) b[j] = 0.0f;
  }
}

int orc_closure_set(orc_ctx* c, const float* params) {
  if (!c->cl_params) c->cl_params = (float*)malloc(sizeof(float) * MLP_NPARAM);
  memcpy(c->cl_params, params, sizeof(float) * MLP_NPARAM);
  return 0;
}

/* X[n][13]: the closure inputs of every cell from moments `which` */
int orc_closure_features(orc_ctx* c, int32_t which, float* X) {
  if (!c->vol) return fail(c, -7, "mesh not loaded");
  const nd_t d = nondim(c);
  double cnt;
  const double* phi = phi_select(c, which, &cnt);
  double* own = (double*)malloc(sizeof(double) * 6 * c->n_tets);
  closure_inputs(c, &d, phi, cnt, X, own, NULL);
  free(own);
  return 0;
}

/* S13 targets: Y[r][8] = HoT of moments `which` (the long-time average) of
 * cell r mod n, normalised like the inputs by the density X[r][0] and
 * temperature X[r][4] of input row r: sigma (xx, yy, xy, xz, yz) / (rho T),
 * q_t / (rho T^{3/2}).  Rows whose input is invalid (zero density or
 * temperature) or whose cell has no particles in `which` are zero. */
int orc_closure_targets(orc_ctx* c, int32_t which, const float* X, int64_t n_rows, float* Y) {
  if (!c->vol) return fail(c, -7, "mesh not loaded");
  const int64_t n = c->n_tets;
  const nd_t d = nondim(c);
  double cnt;
  const double* phi = phi_select(c, which, &cnt);
  double* own = (double*)malloc(sizeof(double) * 6 * n);
  double* H = (double*)malloc(sizeof(double) * 12 * n);
  double* nbar = (double*)malloc(sizeof(double) * n);
  sampled_hot(c, &d, phi, cnt, own, H, nbar);
  for (int64_t r = 0; r < n_rows; ++r) {
    const int64_t t = r % n;
    const double x0 = X[13 * r], x4 = X[13 * r + 4];
    const double* h = H + 12 * t;
    int ok = cnt > 0 && nbar[t] > 0.0 && x0 > 0.0 && x4 > 0.0;
    double y[8];
    if (ok) {
      const double s = x0 * x4, qn = s * sqrt(x4);
      y[0] = h[0] / s; y[1] = h[1] / s; y[2] = h[3] / s; y[3] = h[4] / s; y[4] = h[5] / s;
      y[5] = h[6] / qn; y[6] = h[7] / qn; y[7] = h[8] / qn;
      for (int k = 0; k < 8 && ok; ++k) ok = isfinite(y[k]) && isfinite((float)y[k]);
    }
    for (int k = 0; k < 8; ++k) Y[8 * r + k] = ok ? (float)y[k] : 0.0f;
  }
  free(own); free(H); free(nbar);
  return 0;
}
