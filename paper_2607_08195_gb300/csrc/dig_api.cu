// dig_api.cu -- host side of the C ABI declared in include/dig.h.
//
// Builds the mesh tables on the host (neighbour table, FP64 face planes,
// volumes, boundary-face tangent bases), lays out the caller's device arena,
// and drives the kernels of dig_kernels.cu on the caller's stream.
#include "../../include/dig.h"
#include "dig_internal.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <thread>
#include <vector>

using namespace dig;

namespace {
constexpr double KB = 1.380649e-23;

// FP32 ln/exp of the collision arithmetic, host copy (used for the initial
// (sigma c_r)_max only; the same IEEE steps as the device functions).
float host_ln_f(float x) {
  uint32_t b;
  std::memcpy(&b, &x, 4);
  int e = (int)((b >> 23) & 0xffu) - 127;
  if (e == -127) return -87.3365448f;
  uint32_t mb = (b & 0x7fffffu) | 0x3f800000u;
  float m;
  std::memcpy(&m, &mb, 4);
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
float host_exp_f(float y) {
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
  std::memcpy(&sc, &sb, 4);
  return p * sc;
}

struct Arena {
  char* base = nullptr;
  size_t off = 0;
  template <class T>
  T* take(size_t n) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += n * sizeof(T);
    return p;
  }
};
}  // namespace

struct dig_ctx {
  dig_config cfg{};
  char err[512] = {0};
  cudaStream_t stream = nullptr;
  // host mesh tables
  int64_t n_tets = 0, n_nodes = 0;
  std::vector<double> nodes;
  std::vector<int32_t> tets;
  std::vector<int32_t> nbr;
  std::vector<signed char> nbrf;
  std::vector<Plane64> plane;
  std::vector<float4> plane32;
  std::vector<double> vol, cumvol, fdtv, area, lsqw, vnd, ivnd;
  std::vector<int> fcell, fface, cfid;  // interior faces (synthetic solver)
  std::vector<BFaceDev> bf;
  std::vector<BCDev> bc;
  std::vector<InflowDev> inflow;
  std::vector<dig_bc> bc_host;
  float margin = 0.0f;
  bool mesh_ok = false;
  // device
  bool bound = false;
  Params P{};
  Buf buf[2]{};
  double* dnodes = nullptr;
  int* dtets = nullptr;
  double* mom_out = nullptr;
  int cur = 0;
  int64_t N = 0;
  bool have_particles = false;
  int64_t step = 0;
  int64_t n_ewma = 0, n_win = 0, n_cum = 0, host_steps = 0;
  int tile_cells = 0, stage_cap = 3072, cta_threads = 256;
  float cmax0 = 0.0f;
  cudaEvent_t ev = nullptr;
  cudaGraphExec_t s10_exec = nullptr;  // the synthetic solve as a CUDA graph (see run_s10)
  long long s10_launches = 0;          // kernels in it
  std::vector<cudaEvent_t> tev;  // event pairs around timed cell passes
  CoupleParams C{};
  std::vector<double> bcU, bcT, bcn;
  int64_t flux_steps = 0, n_couple = 0;
  size_t tev_used = 0;
  bool timing = false;
  // learned closure: FP32 master parameters, Adam moments, gradient
  float *cl_p = nullptr, *cl_m = nullptr, *cl_v = nullptr, *cl_g = nullptr;
  double* cl_acc = nullptr;  // [2] loss accumulators
  int* cl_status = nullptr;
  int* fw_status = nullptr;  // set by the tensor-core forward when a wait gave up
  bool cl_set = false;
  int64_t adam_t = 0;
  // the bound arena (checkpoints copy it whole)
  char* arena = nullptr;
  int64_t arena_bytes = 0;
};

static int fail(dig_ctx* c, int code, const char* msg) {
  if (c) std::snprintf(c->err, sizeof c->err, "%s", msg);
  return code;
}

static int cuda_fail(dig_ctx* c, cudaError_t e, const char* where) {
  if (c) std::snprintf(c->err, sizeof c->err, "%s: %s", where, cudaGetErrorString(e));
  return DIG_ERR_CUDA;
}

#define CK(call)                                             \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

// message of the last failed call made without a context (dig_sort_by_cell)
static thread_local char g_err[256] = {0};

static int fail0(int code, const char* msg) {
  std::snprintf(g_err, sizeof g_err, "%s", msg);
  return code;
}

namespace dig {
void set_thread_error(const char* msg) { std::snprintf(g_err, sizeof g_err, "%s", msg); }
}  // namespace dig

extern "C" {

const char* dig_last_error(dig_ctx* ctx) { return ctx ? ctx->err : g_err; }

int dig_create(const dig_config* cfg, dig_ctx** out) {
  if (!cfg || !out) return DIG_ERR_ARG;
  if (!(cfg->mass > 0) || !(cfg->dt > 0) || !(cfg->F_N > 0) || !(cfg->alpha > 0) ||
      (cfg->rot_dof != 0 && cfg->rot_dof != 2) || (cfg->recon != 0 && cfg->recon != 1) ||
      (cfg->local_acc != 0 && cfg->local_acc != 1) || cfg->tile_cells > 2048 ||
      cfg->stage_cap > 8192 || cfg->aa_m < 0 || cfg->aa_m > AA_MAX)
    return DIG_ERR_ARG;
  dig_ctx* c = new dig_ctx();
  c->cfg = *cfg;
  if (c->cfg.max_cross <= 0) c->cfg.max_cross = 4096;
  if (!(c->cfg.wait_timeout_s > 0)) c->cfg.wait_timeout_s = 600.0;
  if (c->cfg.stage_cap > 0) c->stage_cap = c->cfg.stage_cap;
  if (c->cfg.cta_threads > 0) c->cta_threads = c->cfg.cta_threads <= 64 ? 64 : c->cfg.cta_threads <= 128 ? 128 : 256;
  if (c->cfg.n_a <= 0) c->cfg.n_a = 1000;
  if (!(c->cfg.cfl > 0)) c->cfg.cfl = 1.5;
  c->tile_cells = c->cfg.tile_cells;
  *out = c;
  return DIG_OK;
}

int dig_destroy(dig_ctx* ctx) {
  if (!ctx) return DIG_ERR_ARG;
  if (ctx->ev) cudaEventDestroy(ctx->ev);
  if (ctx->s10_exec) cudaGraphExecDestroy(ctx->s10_exec);
  for (cudaEvent_t e : ctx->tev) cudaEventDestroy(e);
  delete ctx;
  return DIG_OK;
}

int dig_set_stream(dig_ctx* ctx, void* s) {
  if (!ctx) return DIG_ERR_ARG;
  ctx->stream = (cudaStream_t)s;
  return DIG_OK;
}

// ---------------------------------------------------------------------------
// mesh
// ---------------------------------------------------------------------------
int mesh_load(dig_ctx* ctx, const double* nodes, int64_t n_nodes, const int32_t* tets, int64_t n_tets,
              const int32_t* face_tag, const dig_bc* bcs, int32_t n_bcs) {
  if (!ctx || !nodes || !tets || !face_tag || n_nodes <= 0 || n_tets <= 0 || n_tets > (1LL << 30))
    return fail(ctx, DIG_ERR_ARG, "mesh_load: bad arguments");
  if (ctx->bound) return fail(ctx, DIG_ERR_STATE, "mesh_load: arena already bound");
  const int64_t n = n_tets;
  ctx->n_tets = n;
  ctx->n_nodes = n_nodes;
  ctx->nodes.assign(nodes, nodes + 3 * n_nodes);
  ctx->tets.assign(tets, tets + 4 * n);
  for (int64_t i = 0; i < 4 * n; ++i)
    if (tets[i] < 0 || tets[i] >= n_nodes) return fail(ctx, DIG_ERR_MESH, "tet vertex index out of range");
  ctx->vol.resize(n);
  ctx->cumvol.resize(n);
  ctx->fdtv.resize(n);
  ctx->plane.resize(4 * n);
  ctx->plane32.resize(4 * n);
  ctx->area.resize(4 * n);
  ctx->nbr.assign(4 * n, INT32_MIN);
  ctx->nbrf.assign(4 * n, 0);
  double run = 0.0, maxd = 0.0, maxx = 0.0;
  for (int64_t i = 0; i < 3 * n_nodes; ++i) maxx = std::max(maxx, std::fabs(nodes[i]));
  for (int64_t t = 0; t < n; ++t) {
    const double* A = nodes + 3 * tets[4 * t + 0];
    const double* B = nodes + 3 * tets[4 * t + 1];
    const double* C = nodes + 3 * tets[4 * t + 2];
    const double* D = nodes + 3 * tets[4 * t + 3];
    double u[3], v[3], w[3];
    for (int i = 0; i < 3; ++i) {
      u[i] = B[i] - A[i];
      v[i] = C[i] - A[i];
      w[i] = D[i] - A[i];
    }
    const double det = u[0] * (v[1] * w[2] - v[2] * w[1]) - u[1] * (v[0] * w[2] - v[2] * w[0]) +
                       u[2] * (v[0] * w[1] - v[1] * w[0]);
    const double V = std::fabs(det) / 6.0;
    if (!(V > 0.0)) return fail(ctx, DIG_ERR_MESH, "degenerate tetrahedron (zero volume)");
    ctx->vol[t] = V;
    run = (t == 0 ? 0.0 : run) + V;
    ctx->cumvol[t] = run;
    ctx->fdtv[t] = ctx->cfg.F_N * ctx->cfg.dt / V;
    for (int f = 0; f < 4; ++f) {
      int lv[3], k = 0;
      for (int q = 0; q < 4; ++q)
        if (q != f) lv[k++] = q;
      const double* a = nodes + 3 * tets[4 * t + lv[0]];
      const double* b = nodes + 3 * tets[4 * t + lv[1]];
      const double* cc = nodes + 3 * tets[4 * t + lv[2]];
      const double* p = nodes + 3 * tets[4 * t + f];
      double e1[3], e2[3], nn[3];
      for (int i = 0; i < 3; ++i) {
        e1[i] = b[i] - a[i];
        e2[i] = cc[i] - a[i];
      }
      nn[0] = e1[1] * e2[2] - e1[2] * e2[1];
      nn[1] = e1[2] * e2[0] - e1[0] * e2[2];
      nn[2] = e1[0] * e2[1] - e1[1] * e2[0];
      const double side = nn[0] * (p[0] - a[0]) + nn[1] * (p[1] - a[1]) + nn[2] * (p[2] - a[2]);
      if (side > 0.0) {
        nn[0] = -nn[0];
        nn[1] = -nn[1];
        nn[2] = -nn[2];
      }
      const double len = std::sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
      ctx->area[4 * t + f] = 0.5 * len;
      nn[0] = nn[0] / len;
      nn[1] = nn[1] / len;
      nn[2] = nn[2] / len;
      const double d = nn[0] * a[0] + nn[1] * a[1] + nn[2] * a[2];
      ctx->plane[4 * t + f] = Plane64{nn[0], nn[1], nn[2], d};
      ctx->plane32[4 * t + f] = make_float4((float)nn[0], (float)nn[1], (float)nn[2], (float)d);
      maxd = std::max(maxd, std::fabs(d));
    }
  }
  // FP32 inside-filter margin: the FP32 plane test d - n.x differs from the
  // exact value by at most ~6 u (|d| + |n|_1 |x|_inf), u = 2^-24; 32 u
  // (max|d| + sqrt3 max|x|) leaves a factor > 2 for particles slightly
  // outside the node bounding box.
  ctx->margin = (float)(32.0 * std::ldexp(1.0, -24) * (maxd + std::sqrt(3.0) * maxx * 1.01));

  // neighbours: faces keyed by their sorted vertex triple
  struct FK {
    int32_t a, b, c, tet, face;
  };
  std::vector<FK> keys(4 * n);
  for (int64_t t = 0; t < n; ++t)
    for (int f = 0; f < 4; ++f) {
      int32_t v3[3], k = 0;
      for (int q = 0; q < 4; ++q)
        if (q != f) v3[k++] = tets[4 * t + q];
      std::sort(v3, v3 + 3);
      keys[4 * t + f] = FK{v3[0], v3[1], v3[2], (int32_t)t, f};
    }
  std::sort(keys.begin(), keys.end(), [](const FK& x, const FK& y) {
    if (x.a != y.a) return x.a < y.a;
    if (x.b != y.b) return x.b < y.b;
    if (x.c != y.c) return x.c < y.c;
    if (x.tet != y.tet) return x.tet < y.tet;
    return x.face < y.face;
  });
  for (size_t i = 0; i < keys.size();) {
    size_t j = i + 1;
    while (j < keys.size() && keys[j].a == keys[i].a && keys[j].b == keys[i].b && keys[j].c == keys[i].c) ++j;
    if (j - i > 2) return fail(ctx, DIG_ERR_MESH, "non-manifold face (shared by more than two tets)");
    if (j - i == 2) {
      const FK& P0 = keys[i];
      const FK& Q0 = keys[i + 1];
      if (face_tag[4 * P0.tet + P0.face] >= 0 || face_tag[4 * Q0.tet + Q0.face] >= 0)
        return fail(ctx, DIG_ERR_MESH, "interior face carries a boundary tag");
      ctx->nbr[4 * P0.tet + P0.face] = Q0.tet;
      ctx->nbrf[4 * P0.tet + P0.face] = (signed char)Q0.face;
      ctx->nbr[4 * Q0.tet + Q0.face] = P0.tet;
      ctx->nbrf[4 * Q0.tet + Q0.face] = (signed char)P0.face;
    } else {
      const int32_t tag = face_tag[4 * keys[i].tet + keys[i].face];
      if (tag < 0 || tag >= n_bcs) return fail(ctx, DIG_ERR_MESH, "boundary face without a valid tag");
    }
    i = j;
  }
  ctx->bc.resize(std::max(1, n_bcs));
  ctx->bc_host.assign(bcs, bcs + n_bcs);
  ctx->bc_host.resize(std::max(1, n_bcs));
  for (int b = 0; b < n_bcs; ++b) {
    BCDev& B = ctx->bc[b];
    B.kind = bcs[b].kind;
    B.sigma = (float)std::sqrt(KB * bcs[b].T / ctx->cfg.mass);
    B.T = (float)bcs[b].T;
    for (int i = 0; i < 3; ++i) B.U[i] = (float)bcs[b].U[i];
  }
  ctx->bf.clear();
  ctx->inflow.clear();
  for (int64_t t = 0; t < n; ++t)
    for (int f = 0; f < 4; ++f) {
      if (ctx->nbr[4 * t + f] != INT32_MIN) continue;
      const Plane64 pl = ctx->plane[4 * t + f];
      const double N3[3] = {pl.nx, pl.ny, pl.nz};
      double a[3] = {1.0, 0.0, 0.0};
      if (std::fabs(N3[0]) >= 0.9) {
        a[0] = 0.0;
        a[1] = 1.0;
      }
      const double an = a[0] * N3[0] + a[1] * N3[1] + a[2] * N3[2];
      double t1[3] = {a[0] - an * N3[0], a[1] - an * N3[1], a[2] - an * N3[2]};
      const double l1 = std::sqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
      t1[0] = t1[0] / l1;
      t1[1] = t1[1] / l1;
      t1[2] = t1[2] / l1;
      const double t2[3] = {N3[1] * t1[2] - N3[2] * t1[1], N3[2] * t1[0] - N3[0] * t1[2],
                            N3[0] * t1[1] - N3[1] * t1[0]};
      BFaceDev B;
      B.bc = face_tag[4 * t + f];
      for (int i = 0; i < 3; ++i) {
        B.nrm[i] = (float)N3[i];
        B.t1[i] = (float)t1[i];
        B.t2[i] = (float)t2[i];
      }
      if (bcs[B.bc].kind == DIG_BC_INFLOW) {
        // Bird (1994) eq. 4.22: one-sided number flux of the drifting free stream
        // through the face, inward normal -n; constants of the inflow law
        const dig_bc& fb = bcs[B.bc];
        InflowDev F{};
        F.bface = (int)ctx->bf.size();
        F.tet = (int)t;
        F.face = f;
        int vq[3], kq = 0;
        for (int q = 0; q < 4; ++q)
          if (q != f) vq[kq++] = tets[4 * t + q];
        const double* P0 = nodes + 3 * vq[0];
        const double* P1 = nodes + 3 * vq[1];
        const double* P2 = nodes + 3 * vq[2];
        double e1[3], e2[3];
        for (int i = 0; i < 3; ++i) {
          F.a[i] = P0[i];
          F.b[i] = P1[i];
          F.c[i] = P2[i];
          e1[i] = P1[i] - P0[i];
          e2[i] = P2[i] - P0[i];
        }
        const double cx = e1[1] * e2[2] - e1[2] * e2[1], cy = e1[2] * e2[0] - e1[0] * e2[2],
                     cz = e1[0] * e2[1] - e1[1] * e2[0];
        const double area = 0.5 * std::sqrt(cx * cx + cy * cy + cz * cz);
        const double beta = std::sqrt(ctx->cfg.mass / (2.0 * KB * fb.T));
        const double sn = -beta * (fb.U[0] * N3[0] + fb.U[1] * N3[1] + fb.U[2] * N3[2]);
        // 1 + erf(s) evaluated as erfc(-s): no cancellation on faces the
        // stream leaves (s << 0)
        const double flux = fb.n / (2.0 * std::sqrt(M_PI) * beta) *
                            (std::exp(-sn * sn) + std::sqrt(M_PI) * sn * std::erfc(-sn));
        F.expn = flux * area * ctx->cfg.dt / ctx->cfg.F_N;
        F.s = (float)sn;
        const double m1 = 0.5, m2 = sn > 0.0 ? sn * std::sqrt(M_PI) : 0.0;
        F.p1 = (float)(m1 / (m1 + m2));
        F.invb = (float)(1.0 / beta);
        F.sig = (float)std::sqrt(KB * fb.T / ctx->cfg.mass);
        F.ut1 = (float)(fb.U[0] * t1[0] + fb.U[1] * t1[1] + fb.U[2] * t1[2]);
        F.ut2 = (float)(fb.U[0] * t2[0] + fb.U[1] * t2[1] + fb.U[2] * t2[2]);
        ctx->inflow.push_back(F);
      }
      ctx->nbr[4 * t + f] = -1 - (int32_t)ctx->bf.size();
      ctx->nbrf[4 * t + f] = (signed char)f;
      ctx->bf.push_back(B);
    }
  // interior faces, each once (from its lower-index cell), for the synthetic solver
  ctx->fcell.clear();
  ctx->fface.clear();
  ctx->cfid.assign(4 * (size_t)n_tets, -1);
  for (int64_t t = 0; t < n_tets; ++t)
    for (int f = 0; f < 4; ++f) {
      const int nb = ctx->nbr[4 * t + f];
      if (nb <= t) continue;
      const int id = (int)ctx->fcell.size();
      ctx->fcell.push_back((int)t);
      ctx->fface.push_back(f);
      ctx->cfid[4 * t + f] = id;
      ctx->cfid[4 * (size_t)nb + ctx->nbrf[4 * t + f]] = id;
    }
  // least-squares gradient weights of every cell (synthetic solver): with
  // d_f = x_f - x_c over the four faces (x_f the neighbour's centroid, or the
  // face centroid at a boundary face; lengths over L_ref) and M = sum d_f d_f^T,
  // grad phi = sum_f (M^-1 d_f) (phi_f - phi_c), exact for linear fields
  ctx->lsqw.assign(12 * (size_t)n_tets, 0.0);
  {
    const double s = 1.0 / ctx->cfg.L_ref;
    auto centroid = [&](int64_t t, double* x) {
      for (int i = 0; i < 3; ++i) {
        double a = 0.0;
        for (int v = 0; v < 4; ++v) a += nodes[3 * (int64_t)tets[4 * t + v] + i];
        x[i] = 0.25 * a * s;
      }
    };
    for (int64_t t = 0; t < n_tets; ++t) {
      double xc[3], d[4][3], M[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
      centroid(t, xc);
      for (int f = 0; f < 4; ++f) {
        const int nb = ctx->nbr[4 * t + f];
        double xf[3];
        if (nb >= 0) {
          centroid(nb, xf);
        } else {
          for (int i = 0; i < 3; ++i) {
            double a = 0.0;
            for (int v = 0; v < 4; ++v)
              if (v != f) a += nodes[3 * (int64_t)tets[4 * t + v] + i];
            xf[i] = a / 3.0 * s;
          }
        }
        for (int i = 0; i < 3; ++i) d[f][i] = xf[i] - xc[i];
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) M[i][j] += d[f][i] * d[f][j];
      }
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
      if (!(std::fabs(det) > 0.0)) return fail(ctx, DIG_ERR_MESH, "degenerate least-squares stencil");
      for (int f = 0; f < 4; ++f)
        for (int i = 0; i < 3; ++i)
          ctx->lsqw[(size_t)(3 * f + i) * n_tets + t] =
              (A[i][0] * d[f][0] + A[i][1] * d[f][1] + A[i][2] * d[f][2]) / det;
    }
  }
  ctx->mesh_ok = true;
  return DIG_OK;
}

// ---------------------------------------------------------------------------
// arena
// ---------------------------------------------------------------------------
static size_t layout(dig_ctx* ctx, char* base) {
  Arena A;
  A.base = base;
  const size_t n = (size_t)ctx->n_tets, cap = (size_t)ctx->cfg.capacity, nb = ctx->bf.size();
  Params& P = ctx->P;
  P.nbr = A.take<int>(4 * n);
  P.nbrf = A.take<signed char>(4 * n);
  P.plane = A.take<Plane64>(4 * n);
  P.plane32 = A.take<float4>(4 * n);
  P.fdtv = A.take<double>(n);
  P.vol = A.take<double>(n);
  P.cumvol = A.take<double>(n);
  P.bf = A.take<BFaceDev>(std::max<size_t>(nb, 1));
  P.bc = A.take<BCDev>(ctx->bc.size());
  P.bflux = A.take<double>(5 * std::max<size_t>(nb, 1));
  const size_t ni = ctx->inflow.size();
  P.inflow = A.take<InflowDev>(std::max<size_t>(ni, 1));
  P.inj_rem = A.take<double>(std::max<size_t>(ni, 1));
  P.inj_cnt = A.take<int>(std::max<size_t>(ni, 1));
  P.inj_off = A.take<int>(ni + 1);
  ctx->dnodes = A.take<double>(3 * (size_t)ctx->n_nodes);
  ctx->dtets = A.take<int>(4 * n);
  P.nodes = ctx->dnodes;
  P.tets = ctx->dtets;
  for (int b = 0; b < 2; ++b) {
    double* xs = A.take<double>(3 * cap);
    float* vs = A.take<float>(3 * cap);
    float* Is = A.take<float>(cap);
    int* mc = A.take<int>(cap);
    ctx->buf[b] = Buf{xs, vs, Is, mc};
  }
  P.cs = A.take<int>(n + 1);
  P.as = A.take<int>(n + 1);
  P.nst = A.take<int>(n);
  P.sbase = A.take<int>(n);
  P.nold = A.take<int>(n);
  P.na = A.take<int>(n);
  P.fill = A.take<int>(n);
  P.aq = A.take<int>(cap);
  P.tq = A.take<int>(2 * cap);
  P.src = A.take<int>(cap);
  P.cmax = A.take<float>(n);
  P.rem = A.take<double>(n);
  P.phi_inst = A.take<double>(NPHI * n);
  P.phi_ewma = A.take<double>(NPHI * n);
  P.phi_win = A.take<double>(NPHI * n);
  P.phi_cum = A.take<double>(NPHI * n);
  P.acc_w = A.take<double>(n);
  ctx->mom_out = A.take<double>(NMAC * n);
  P.counters = A.take<unsigned long long>(16);
  P.status = A.take<int>(4);
  P.state = A.take<int>(8);
  P.scan_part = A.take<int>(2 * (size_t)scan_blocks((int)n) + 2);
  P.pair_cap = (long long)std::max<size_t>(cap, 1 << 16);
  P.pairs = A.take<int>(4 * (size_t)P.pair_cap);
  P.pacc = A.take<unsigned char>((size_t)P.pair_cap);
  P.pair_count = A.take<unsigned long long>(1);
  // DIG coupling
  CoupleParams& C = ctx->C;
  C.area = A.take<double>(4 * n);
  C.lsqw = A.take<double>(12 * n);
  C.vnd = A.take<double>(n);
  C.ivnd = A.take<double>(n);
  const size_t nbc = std::max<size_t>(ctx->bc.size(), 1);
  C.bcU = A.take<double>(3 * nbc);
  C.bcT = A.take<double>(nbc);
  C.bcn = A.take<double>(nbc);
  C.own = A.take<double>(6 * n);
  C.sd = A.take<double>(12 * n);
  C.grad = A.take<double>(15 * n);
  C.half = A.take<double>(6 * n);
  C.hot = A.take<double>(12 * n);
  C.newst = A.take<double>(6 * n);
  C.flag = A.take<double>(n);
  C.nbar = A.take<double>(n);
  C.U = A.take<double>(6 * n);
  C.prim = A.take<double>(6 * n);
  C.S = A.take<double>(12 * n);
  C.R = A.take<double>(6 * n);
  C.mu = A.take<double>(n);
  C.snd = A.take<double>(n);
  C.mach = A.take<double>(n);
  const size_t nif = std::max<size_t>(ctx->fcell.size(), 1);
  C.fcell = A.take<int>(nif);
  C.fface = A.take<int>(nif);
  C.cfid = A.take<int>(4 * n);
  C.Ff = A.take<double>(6 * nif);
  C.lmf = A.take<double>(nif);
  C.part = A.take<double>(couple_part_count((int)n));
  C.dtl = A.take<double>(n);
  C.fp = A.take<double>(6 * n);
  C.Gp = A.take<double>(6 * n);
  C.Ub = A.take<double>(6 * n);
  const size_t naa = (size_t)std::max(ctx->cfg.aa_m, 1);
  C.dF = A.take<double>(naa * 6 * n);
  C.dG = A.take<double>(naa * 6 * n);
  C.apart = A.take<double>(couple_apart_count((int)n));
  C.aab = couple_aa_blocks((int)n);
  C.aa = A.take<AAState>(1);
  C.avail = A.take<int>(n);
  C.avail2 = A.take<int>(n);
  C.feat = A.take<float>((size_t)MLP_NIN * n);
  C.ypred = A.take<float>((size_t)MLP_NOUT * n);
  C.wnorm = A.take<double>(2 * n);
  C.stats = A.take<unsigned long long>(8);
  C.fillcnt = A.take<int>(DIG_FILL_LAYERS);
  ctx->cl_p = A.take<float>(MLP_NPARAM);
  ctx->cl_m = A.take<float>(MLP_NPARAM);
  ctx->cl_v = A.take<float>(MLP_NPARAM);
  ctx->cl_g = A.take<float>(MLP_NPARAM);
  ctx->cl_acc = A.take<double>(2);
  ctx->cl_status = A.take<int>(2);
  ctx->fw_status = A.take<int>(1);
  C.scal = A.take<CoupleScalars>(1);
  C.rpart = A.take<int>(cap / 4096 + 2);
  C.clone_total = A.take<int>(1);
  return A.off + 256;
}

int dig_arena_bytes(dig_ctx* ctx, int64_t* bytes) {
  if (!ctx || !bytes) return DIG_ERR_ARG;
  if (!ctx->mesh_ok) return fail(ctx, DIG_ERR_STATE, "dig_arena_bytes: no mesh loaded");
  if (ctx->cfg.capacity <= 0 || ctx->cfg.capacity > (1LL << 31) - 64)
    return fail(ctx, DIG_ERR_ARG, "capacity must be in [1, 2^31 - 64]");
  *bytes = (int64_t)layout(ctx, nullptr);
  return DIG_OK;
}

int dig_bind_arena(dig_ctx* ctx, void* dptr, int64_t bytes) {
  if (!ctx || !dptr) return DIG_ERR_ARG;
  if (!ctx->mesh_ok) return fail(ctx, DIG_ERR_STATE, "dig_bind_arena: no mesh loaded");
  if (((uintptr_t)dptr & 255) != 0) return fail(ctx, DIG_ERR_ARG, "arena must be 256-byte aligned");
  if (ctx->s10_exec) {  // captured with the previous arena's pointers
    cudaGraphExecDestroy(ctx->s10_exec);
    ctx->s10_exec = nullptr;
  }
  int64_t need = 0;
  int rc = dig_arena_bytes(ctx, &need);
  if (rc) return rc;
  if (bytes < need) return fail(ctx, DIG_ERR_CAPACITY, "arena smaller than dig_arena_bytes()");
  layout(ctx, (char*)dptr);
  ctx->arena = (char*)dptr;
  ctx->arena_bytes = need;
  Params& P = ctx->P;
  const dig_config& c = ctx->cfg;
  const size_t n = (size_t)ctx->n_tets;
  P.n_cells = (int)n;
  P.n_bf = (int)ctx->bf.size();
  P.n_in = (int)ctx->inflow.size();
  P.max_cross = c.max_cross;
  P.rot_dof = c.rot_dof;
  P.margin = ctx->margin;
  P.dt = c.dt;
  P.mass_fn = c.mass * c.F_N;
  P.fn_kb = c.F_N * KB;
  P.seed_lo = (uint32_t)c.seed;
  P.seed_hi = (uint32_t)(c.seed >> 32);
  const double m = c.mass, w = c.omega, mr = 0.5 * m;
  P.c_vhs = (float)(M_PI * c.d_ref * c.d_ref * std::pow(2.0 * KB * c.T_ref / mr, w - 0.5) / std::tgamma(2.5 - w));
  P.one_m_omega = (float)(1.0 - w);
  const float c0sq = (float)(6.25 * 2.0 * KB * c.T_init / m);
  ctx->cmax0 = P.c_vhs * host_exp_f(P.one_m_omega * host_ln_f(c0sq));
  const double a = c.alpha;
  P.p_inel = (float)(a * (5.0 - 2.0 * w) * (7.0 - 2.0 * w) / (5.0 * (a + 1.0) * (a + 2.0) * c.Z_rot));
  P.vss = a != 1.0 ? 1 : 0;
  P.inv_alpha = (float)(1.0 / a);
  P.lb_exp = (float)(1.0 / (2.5 - w));
  P.hmr = (float)(0.5 * mr / KB);
  P.T_init = (float)c.T_init;
  P.sigma_init = (float)std::sqrt(KB * c.T_init / m);
  for (int i = 0; i < 3; ++i) P.u0[i] = (float)c.u_init[i];
  P.cap = c.capacity;
  cudaStream_t s = ctx->stream;
  CK(cudaMemcpyAsync((void*)P.nbr, ctx->nbr.data(), 4 * n * sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync((void*)P.nbrf, ctx->nbrf.data(), 4 * n, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync((void*)P.plane, ctx->plane.data(), 4 * n * sizeof(Plane64), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync((void*)P.plane32, ctx->plane32.data(), 4 * n * sizeof(float4), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync((void*)P.fdtv, ctx->fdtv.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync((void*)P.vol, ctx->vol.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync((void*)P.cumvol, ctx->cumvol.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
  if (!ctx->bf.empty())
    CK(cudaMemcpyAsync((void*)P.bf, ctx->bf.data(), ctx->bf.size() * sizeof(BFaceDev), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync((void*)P.bc, ctx->bc.data(), ctx->bc.size() * sizeof(BCDev), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(P.bflux, 0, 5 * std::max<size_t>(ctx->bf.size(), 1) * sizeof(double), s));
  if (!ctx->inflow.empty()) {
    CK(cudaMemcpyAsync((void*)P.inflow, ctx->inflow.data(), ctx->inflow.size() * sizeof(InflowDev),
                       cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(P.inj_rem, 0, ctx->inflow.size() * sizeof(double), s));
  }
  CK(cudaMemcpyAsync(ctx->dnodes, ctx->nodes.data(), ctx->nodes.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(ctx->dtets, ctx->tets.data(), ctx->tets.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  std::vector<float> cm(n, ctx->cmax0);
  CK(cudaMemcpyAsync(P.cmax, cm.data(), n * sizeof(float), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(P.rem, 0, n * sizeof(double), s));
  for (double* ph : {P.phi_inst, P.phi_ewma, P.phi_win, P.phi_cum})
    CK(cudaMemsetAsync(ph, 0, NPHI * n * sizeof(double), s));
  CK(cudaMemsetAsync(P.acc_w, 0, n * sizeof(double), s));
  P.local_acc = c.local_acc;
  CK(cudaMemsetAsync(P.counters, 0, 16 * sizeof(unsigned long long), s));
  CK(cudaMemsetAsync(P.status, 0, 4 * sizeof(int), s));
  CK(cudaMemsetAsync(P.state, 0, 8 * sizeof(int), s));
  CK(cudaMemsetAsync(P.cs, 0, (n + 1) * sizeof(int), s));
  CK(cudaMemsetAsync(P.as, 0, (n + 1) * sizeof(int), s));
  for (int* q : {P.nst, P.sbase, P.nold, P.na, P.fill}) CK(cudaMemsetAsync(q, 0, n * sizeof(int), s));
  CK(cudaMemsetAsync(P.pair_count, 0, sizeof(unsigned long long), s));
  // no slot refers to a cell until a pass writes it
  for (int b = 0; b < 2; ++b) CK(cudaMemsetAsync(ctx->buf[b].mc, 0xff, (size_t)c.capacity * sizeof(int), s));
  {
    CoupleParams& C = ctx->C;
    CK(cudaMemcpyAsync((void*)C.area, ctx->area.data(), 4 * n * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync((void*)C.lsqw, ctx->lsqw.data(), 12 * n * sizeof(double), cudaMemcpyHostToDevice, s));
    {
      const double L3 = c.L_ref * c.L_ref * c.L_ref;
      ctx->vnd.resize(n);
      ctx->ivnd.resize(n);
      for (size_t t = 0; t < n; ++t) {
        ctx->vnd[t] = ctx->vol[t] / L3;
        ctx->ivnd[t] = L3 / ctx->vol[t];
      }
      CK(cudaMemcpyAsync((void*)C.vnd, ctx->vnd.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
      CK(cudaMemcpyAsync((void*)C.ivnd, ctx->ivnd.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
    }
    C.n_ifaces = (int)ctx->fcell.size();
    if (C.n_ifaces > 0) {
      CK(cudaMemcpyAsync((void*)C.fcell, ctx->fcell.data(), C.n_ifaces * sizeof(int), cudaMemcpyHostToDevice, s));
      CK(cudaMemcpyAsync((void*)C.fface, ctx->fface.data(), C.n_ifaces * sizeof(int), cudaMemcpyHostToDevice, s));
    }
    CK(cudaMemcpyAsync((void*)C.cfid, ctx->cfid.data(), 4 * n * sizeof(int), cudaMemcpyHostToDevice, s));
    ctx->bcU.assign(3 * ctx->bc.size(), 0.0);
    ctx->bcT.assign(ctx->bc.size(), 0.0);
    ctx->bcn.assign(ctx->bc.size(), 0.0);
    for (size_t b = 0; b < ctx->bc.size(); ++b) {
      for (int i = 0; i < 3; ++i) ctx->bcU[3 * b + i] = ctx->bc_host[b].U[i];
      ctx->bcT[b] = ctx->bc_host[b].T;
      ctx->bcn[b] = ctx->bc_host[b].n;
    }
    if (!ctx->bc.empty()) {
      CK(cudaMemcpyAsync((void*)C.bcU, ctx->bcU.data(), ctx->bcU.size() * sizeof(double), cudaMemcpyHostToDevice, s));
      CK(cudaMemcpyAsync((void*)C.bcT, ctx->bcT.data(), ctx->bcT.size() * sizeof(double), cudaMemcpyHostToDevice, s));
      CK(cudaMemcpyAsync((void*)C.bcn, ctx->bcn.data(), ctx->bcn.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    }
    C.L0 = c.L_ref;
    C.iL2 = 1.0 / (c.L_ref * c.L_ref);
    C.T0 = c.T_init;
    C.rho0 = c.mass * c.n_init;
    C.c0 = std::sqrt(KB / c.mass * C.T0);
    for (int i = 0; i < 3; ++i) C.u_ref[i] = c.u_init[i] / C.c0;
    C.Kn = c.Kn;
    C.omega = c.omega;
    C.dr = (double)c.rot_dof;
    C.gam = (5.0 + C.dr) / (3.0 + C.dr);
    C.Zr = c.Z_rot;
    C.mass = c.mass;
    C.FN = c.F_N;
    C.kB = KB;
    C.KnD_max = c.KnD_max;
    C.recon = c.recon;
    C.N_m = c.N_m;
    C.eps_m = c.eps_m;
    C.aa_m = c.aa_m;
    C.cfl = c.cfl;
    C.closed = 1;
    for (const dig_bc& b : ctx->bc_host)
      if (b.kind == DIG_BC_INFLOW || b.kind == DIG_BC_OUTFLOW) C.closed = 0;
  }
  CK(cudaStreamSynchronize(s));
  if (!ctx->ev) CK(cudaEventCreateWithFlags(&ctx->ev, cudaEventDisableTiming));
  ctx->bound = true;
  return DIG_OK;
}

// ---------------------------------------------------------------------------
// waits and status
// ---------------------------------------------------------------------------
static int check_forward(dig_ctx* ctx);

static int wait_stream(dig_ctx* ctx) {
  CK(cudaEventRecord(ctx->ev, ctx->stream));
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaEventQuery(ctx->ev);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) return cuda_fail(ctx, e, "waiting for the stream");
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (el > ctx->cfg.wait_timeout_s) return fail(ctx, DIG_ERR_TIMEOUT, "host wait on the stream timed out");
    std::this_thread::sleep_for(std::chrono::microseconds(el < 0.01 ? 5 : 200));
  }
  return DIG_OK;
}

static int check_status(dig_ctx* ctx) {
  int st[4] = {0, 0, 0, 0};
  unsigned long long cnt[16];
  CK(cudaMemcpyAsync(st, ctx->P.status, sizeof st, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(cnt, ctx->P.counters, sizeof cnt, cudaMemcpyDeviceToHost, ctx->stream));
  int rc = wait_stream(ctx);
  if (rc) return rc;
  if (st[0] & ST_CAPACITY) return fail(ctx, DIG_ERR_CAPACITY, "particle count exceeded the capacity");
  if (cnt[C_STUCK] > 0) return fail(ctx, DIG_ERR_STUCK, "particles exceeded the face-crossing limit");
  return DIG_OK;
}

int dig_synchronize(dig_ctx* ctx) {
  if (!ctx) return DIG_ERR_ARG;
  if (!ctx->bound) return wait_stream(ctx);
  return check_status(ctx);
}

// ---------------------------------------------------------------------------
// particle loop
// ---------------------------------------------------------------------------
static void choose_tile(dig_ctx* ctx) {
  if (ctx->cfg.tile_cells > 0) {
    ctx->tile_cells = ctx->cfg.tile_cells;
    return;
  }
  const double mean = std::max(1.0, (double)ctx->N / (double)ctx->n_tets);
  int tc = (int)(0.75 * ctx->stage_cap / mean);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int by_grid = (int)((ctx->n_tets + 2 * sms - 1) / (2 * sms));
  tc = std::min(tc, std::max(1, by_grid));
  ctx->tile_cells = std::max(1, std::min(tc, 256));
}

// one gather/collide/move pass followed by the counting-sort bookkeeping
static cudaEvent_t timing_event(dig_ctx* ctx) {
  if (ctx->tev_used == ctx->tev.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    ctx->tev.push_back(e);
  }
  return ctx->tev[ctx->tev_used++];
}

// ewa, ewb: weights of the moving average for this step, avg = ewa avg + ewb sample
static void pass(dig_ctx* ctx, int pass_flags, int sflags, uint32_t step_coll, uint32_t step_move, double ewa,
                 double ewb) {
  const int other = 1 - ctx->cur;
  if (ctx->timing) cudaEventRecord(timing_event(ctx), ctx->stream);
  launch_cell_pass(ctx->P, ctx->buf[ctx->cur], ctx->buf[other], pass_flags, sflags, step_coll, step_move,
                   ewa, ewb, ctx->tile_cells, ctx->cta_threads, ctx->stream);
  if (ctx->timing) cudaEventRecord(timing_event(ctx), ctx->stream);
  if (pass_flags & PASS_MOVE)
    launch_inject(ctx->P, ctx->buf[other], step_move, (sflags & S_WALLFLUX) != 0, ctx->stream);
  ctx->cur = other;
  launch_scan(ctx->P, ctx->stream);
  launch_scatter(ctx->P, ctx->buf[ctx->cur].mc, ctx->stream);
}

// particles just written as arrivals into buf[cur] slots [0, n): sort them
static int settle_new_particles(dig_ctx* ctx, int64_t n) {
  ctx->N = n;
  choose_tile(ctx);
  launch_scan(ctx->P, ctx->stream);
  launch_scatter(ctx->P, ctx->buf[ctx->cur].mc, ctx->stream);
  // the first cell pass reads only arrivals (no stayers): gather into the other buffer
  pass(ctx, 0, 0, 0, 0, 0.0, 1.0);
  ctx->have_particles = true;
  return DIG_OK;
}

static int reset_grouping(dig_ctx* ctx, int64_t n) {
  Params& P = ctx->P;
  const size_t nc = (size_t)ctx->n_tets;
  cudaStream_t s = ctx->stream;
  for (int* q : {P.nst, P.sbase, P.nold, P.na, P.fill}) CK(cudaMemsetAsync(q, 0, nc * sizeof(int), s));
  int st[3] = {0, 0, (int)n};
  CK(cudaMemcpyAsync(P.state, st, sizeof st, cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  return DIG_OK;
}

int particles_init(dig_ctx* ctx, int64_t n) {
  if (!ctx) return DIG_ERR_ARG;
  if (!ctx->bound) return fail(ctx, DIG_ERR_STATE, "particles_init: no arena bound");
  if (n < 0 || n > ctx->cfg.capacity) return fail(ctx, DIG_ERR_CAPACITY, "particles_init: n exceeds capacity");
  int rc = reset_grouping(ctx, n);
  if (rc) return rc;
  launch_init(ctx->P, ctx->buf[ctx->cur], (int)n, ctx->stream);
  return settle_new_particles(ctx, n);
}

int write_particles(dig_ctx* ctx, const double* x, const float* v, const float* Ir, const int32_t* cell,
                    int64_t n) {
  if (!ctx || (n > 0 && (!x || !v || !cell))) return DIG_ERR_ARG;
  if (!ctx->bound) return fail(ctx, DIG_ERR_STATE, "write_particles: no arena bound");
  if (n < 0 || n > ctx->cfg.capacity) return fail(ctx, DIG_ERR_CAPACITY, "write_particles: n exceeds capacity");
  for (int64_t p = 0; p < n; ++p)
    if (cell[p] < 0 || cell[p] >= ctx->n_tets) return fail(ctx, DIG_ERR_ARG, "write_particles: cell out of range");
  int rc = reset_grouping(ctx, n);
  if (rc) return rc;
  const Buf& st = ctx->buf[1 - ctx->cur];  // staging in the other buffer
  cudaStream_t s = ctx->stream;
  if (n > 0) {
    CK(cudaMemcpyAsync(st.pos, x, 3 * n * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(st.vel, v, 3 * n * sizeof(float), cudaMemcpyHostToDevice, s));
    if (Ir) CK(cudaMemcpyAsync(st.Ir, Ir, n * sizeof(float), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->P.aq, cell, n * sizeof(int), cudaMemcpyHostToDevice, s));
  }
  launch_write(ctx->P, ctx->buf[ctx->cur], st.pos, st.vel, Ir ? st.Ir : nullptr, ctx->P.aq, (int)n, s);
  return settle_new_particles(ctx, n);
}

int read_particles(dig_ctx* ctx, double* x, float* v, float* Ir, int32_t* cell, int64_t cap, int64_t* n) {
  if (!ctx || !n) return DIG_ERR_ARG;
  if (!ctx->have_particles) {
    *n = 0;
    return DIG_OK;
  }
  int N = 0;
  CK(cudaMemcpyAsync(&N, ctx->P.state, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  int rc = wait_stream(ctx);
  if (rc) return rc;
  *n = N;
  ctx->N = N;
  if (cap < N) return fail(ctx, DIG_ERR_CAPACITY, "read_particles: buffer too small");
  const Buf& st = ctx->buf[1 - ctx->cur];
  cudaStream_t s = ctx->stream;
  launch_read(ctx->P, ctx->buf[ctx->cur], st.pos, st.vel, st.Ir, ctx->P.aq, N, s);
  if (N > 0) {
    if (x) CK(cudaMemcpyAsync(x, st.pos, 3 * (size_t)N * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (v) CK(cudaMemcpyAsync(v, st.vel, 3 * (size_t)N * sizeof(float), cudaMemcpyDeviceToHost, s));
    if (Ir) CK(cudaMemcpyAsync(Ir, st.Ir, (size_t)N * sizeof(float), cudaMemcpyDeviceToHost, s));
    if (cell) CK(cudaMemcpyAsync(cell, ctx->P.aq, (size_t)N * sizeof(int), cudaMemcpyDeviceToHost, s));
  }
  return wait_stream(ctx);
}

int dsmc_step(dig_ctx* ctx, int32_t n_steps, int32_t flags) {
  if (!ctx || n_steps < 0) return DIG_ERR_ARG;
  if (!ctx->have_particles) return fail(ctx, DIG_ERR_STATE, "dsmc_step: no particles");
  if (n_steps == 0) return DIG_OK;
  const int sflags = flags & (S_EWMA | S_WINDOW | S_CUMUL | S_INST | S_WALLFLUX);
  const uint32_t t0 = (uint32_t)ctx->step;
  ctx->timing = (flags & DIG_TIMING) != 0;
  for (int s = 0; s <= n_steps; ++s) {
    int pf = 0, sf = 0;
    double ewa = 0.0, ewb = 1.0;
    if (s > 0) {
      pf |= PASS_COLLIDE;
      sf = sflags & ~S_WALLFLUX;
      if ((flags & DIG_RECORD_PAIRS) && s == n_steps) {
        CK(cudaMemsetAsync(ctx->P.pair_count, 0, sizeof(unsigned long long), ctx->stream));
        sf |= S_PAIRS;
      }
      if (sflags & S_EWMA) {
        // Eq. exponential_average_moments with n_a effective samples; while
        // fewer than n_a samples exist, the plain mean of all of them
        const double m = (double)(ctx->n_ewma + 1), na = (double)ctx->cfg.n_a;
        const double w = m < na ? m : na;
        ewa = (w - 1.0) / w;
        ewb = 1.0 / w;
      }
    }
    if (s < n_steps) {
      pf |= PASS_MOVE;
      sf |= sflags & S_WALLFLUX;
    }
    pass(ctx, pf, sf, t0 + (uint32_t)s, t0 + (uint32_t)s + 1, ewa, ewb);
    if (s > 0) {
      if (sflags & S_EWMA) ctx->n_ewma++;
      if (sflags & S_WINDOW) ctx->n_win++;
      if (sflags & S_CUMUL) ctx->n_cum++;
    }
  }
  ctx->timing = false;
  if (flags & DIG_WALLFLUX) ctx->flux_steps += n_steps;
  ctx->step += n_steps;
  ctx->host_steps += n_steps;
  if (flags & DIG_SYNC) return check_status(ctx);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "dsmc_step launch");
  return DIG_OK;
}

int sample(dig_ctx* ctx, int32_t action) {
  if (!ctx || !ctx->bound) return DIG_ERR_STATE;
  const size_t m = NPHI * (size_t)ctx->n_tets * sizeof(double);
  if (action & DIG_RESET_WINDOW) {
    CK(cudaMemsetAsync(ctx->P.phi_win, 0, m, ctx->stream));
    ctx->n_win = 0;
  }
  if (action & DIG_RESET_CUMUL) {
    CK(cudaMemsetAsync(ctx->P.phi_cum, 0, m, ctx->stream));
    ctx->n_cum = 0;
  }
  if (action & DIG_RESET_EWMA) {
    CK(cudaMemsetAsync(ctx->P.phi_ewma, 0, m, ctx->stream));
    CK(cudaMemsetAsync(ctx->P.acc_w, 0, (size_t)ctx->n_tets * sizeof(double), ctx->stream));
    ctx->n_ewma = 0;
  }
  return DIG_OK;
}

int read_moments(dig_ctx* ctx, int32_t which, double* out, int64_t cap) {
  if (!ctx || !out) return DIG_ERR_ARG;
  if (!ctx->bound) return fail(ctx, DIG_ERR_STATE, "read_moments: no arena");
  const int base = which & 15, macro = (which & DIG_MACRO) != 0;
  const int64_t need = (macro ? NMAC : NPHI) * ctx->n_tets;
  if (cap < need) return fail(ctx, DIG_ERR_CAPACITY, "read_moments: buffer too small");
  const double* src = base == DIG_PHI_INST ? ctx->P.phi_inst
                    : base == DIG_PHI_EWMA ? ctx->P.phi_ewma
                    : base == DIG_PHI_WINDOW ? ctx->P.phi_win : ctx->P.phi_cum;
  double cnt = base == DIG_PHI_WINDOW ? (double)ctx->n_win : base == DIG_PHI_CUM ? (double)ctx->n_cum : 1.0;
  const double scale = (macro && cnt > 0) ? 1.0 / cnt : (macro ? 0.0 : 1.0);
  launch_moments_ex(ctx->P, src, scale, macro, ctx->mom_out, ctx->cfg.mass, ctx->cfg.F_N, KB, ctx->stream);
  CK(cudaMemcpyAsync(out, ctx->mom_out, need * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  return wait_stream(ctx);
}

int read_pairs(dig_ctx* ctx, int32_t* cell, int32_t* k, int32_t* i, int32_t* j, uint8_t* acc, int64_t cap,
               int64_t* n) {
  if (!ctx || !n) return DIG_ERR_ARG;
  unsigned long long cnt = 0;
  CK(cudaMemcpyAsync(&cnt, ctx->P.pair_count, sizeof cnt, cudaMemcpyDeviceToHost, ctx->stream));
  int rc = wait_stream(ctx);
  if (rc) return rc;
  *n = (int64_t)cnt;
  if (cnt > (unsigned long long)ctx->P.pair_cap) return fail(ctx, DIG_ERR_CAPACITY, "pair record overflowed");
  if (!cell || !k || !i || !j || !acc) return DIG_OK;  // size query
  if (cap < (int64_t)cnt) return fail(ctx, DIG_ERR_CAPACITY, "read_pairs: buffer too small");
  std::vector<int32_t> r(4 * cnt);
  std::vector<uint8_t> a(cnt);
  if (cnt) {
    CK(cudaMemcpyAsync(r.data(), ctx->P.pairs, 4 * cnt * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(a.data(), ctx->P.pacc, cnt, cudaMemcpyDeviceToHost, ctx->stream));
  }
  rc = wait_stream(ctx);
  if (rc) return rc;
  std::vector<int64_t> ord(cnt);
  for (size_t q = 0; q < cnt; ++q) ord[q] = (int64_t)q;
  std::sort(ord.begin(), ord.end(), [&](int64_t x, int64_t y) {
    if (r[4 * x] != r[4 * y]) return r[4 * x] < r[4 * y];
    return r[4 * x + 1] < r[4 * y + 1];
  });
  for (size_t q = 0; q < cnt; ++q) {
    const int64_t o = ord[q];
    cell[q] = r[4 * o];
    k[q] = r[4 * o + 1];
    i[q] = r[4 * o + 2];
    j[q] = r[4 * o + 3];
    acc[q] = a[o];
  }
  return DIG_OK;
}

int read_counters(dig_ctx* ctx, int64_t* out, int32_t n) {
  if (!ctx || !out) return DIG_ERR_ARG;
  unsigned long long cnt[16];
  CK(cudaMemcpyAsync(cnt, ctx->P.counters, sizeof cnt, cudaMemcpyDeviceToHost, ctx->stream));
  int rc = wait_stream(ctx);
  if (rc) return rc;
  cnt[C_STEPS] = (unsigned long long)ctx->host_steps;
  for (int q = 0; q < n && q < N_COUNTERS; ++q) out[q] = (int64_t)cnt[q];
  return DIG_OK;
}

int dig_cell_state(dig_ctx* ctx, float* cmax, double* rem, int32_t write) {
  if (!ctx || !ctx->bound) return DIG_ERR_STATE;
  const size_t n = (size_t)ctx->n_tets;
  cudaStream_t s = ctx->stream;
  if (write) {
    if (cmax) CK(cudaMemcpyAsync(ctx->P.cmax, cmax, n * sizeof(float), cudaMemcpyHostToDevice, s));
    if (rem) CK(cudaMemcpyAsync(ctx->P.rem, rem, n * sizeof(double), cudaMemcpyHostToDevice, s));
  } else {
    if (cmax) CK(cudaMemcpyAsync(cmax, ctx->P.cmax, n * sizeof(float), cudaMemcpyDeviceToHost, s));
    if (rem) CK(cudaMemcpyAsync(rem, ctx->P.rem, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  return wait_stream(ctx);
}

int dig_wall_flux(dig_ctx* ctx, double* out, int64_t cap, int64_t* n_bfaces) {
  if (!ctx || !n_bfaces) return DIG_ERR_ARG;
  *n_bfaces = (int64_t)ctx->bf.size();
  if (!ctx->bound) return fail(ctx, DIG_ERR_STATE, "no arena");
  if (!out) return DIG_OK;  // size query
  if (cap < 5 * *n_bfaces) return fail(ctx, DIG_ERR_CAPACITY, "dig_wall_flux: buffer too small");
  CK(cudaMemcpyAsync(out, ctx->P.bflux, 5 * ctx->bf.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  return wait_stream(ctx);
}

int dig_surface(dig_ctx* ctx, double* out, int64_t cap, int64_t* n_bfaces) {
  if (!ctx || !n_bfaces) return DIG_ERR_ARG;
  const size_t nb = ctx->bf.size();
  *n_bfaces = (int64_t)nb;
  if (!ctx->bound) return fail(ctx, DIG_ERR_STATE, "no arena");
  if (!out) return DIG_OK;  // size query
  if (cap < 6 * (int64_t)nb) return fail(ctx, DIG_ERR_CAPACITY, "dig_surface: buffer too small");
  if (ctx->flux_steps <= 0) return fail(ctx, DIG_ERR_STATE, "dig_surface: no steps sampled with DIG_WALLFLUX");
  std::vector<double> F(5 * std::max<size_t>(nb, 1));
  CK(cudaMemcpyAsync(F.data(), ctx->P.bflux, 5 * nb * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  int rc = wait_stream(ctx);
  if (rc) return rc;
  const double t = (double)ctx->flux_steps * ctx->cfg.dt;
  for (int64_t tt = 0; tt < ctx->n_tets; ++tt)
    for (int f = 0; f < 4; ++f) {
      const int32_t code = ctx->nbr[4 * tt + f];
      if (code >= 0) continue;
      const size_t ib = (size_t)(-1 - code);
      const Plane64 pl = ctx->plane[4 * tt + f];  // outward normal of the gas cell: into the wall
      const double At = ctx->area[4 * tt + f] * t;
      const double* G = F.data() + 5 * ib;
      const double gx = G[1] / At, gy = G[2] / At, gz = G[3] / At;
      const double p = gx * pl.nx + gy * pl.ny + gz * pl.nz;
      double* o = out + 6 * ib;
      o[0] = G[0] * ctx->cfg.F_N / At;
      o[1] = p;
      o[2] = gx - p * pl.nx;
      o[3] = gy - p * pl.ny;
      o[4] = gz - p * pl.nz;
      o[5] = G[4] / At;
    }
  return DIG_OK;
}

int dig_particle_count(dig_ctx* ctx, int64_t* n) {
  if (!ctx || !n) return DIG_ERR_ARG;
  if (!ctx->have_particles) {
    *n = 0;
    return DIG_OK;
  }
  int N = 0;
  CK(cudaMemcpyAsync(&N, ctx->P.state, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  int rc = wait_stream(ctx);
  *n = N;
  return rc;
}

int dig_kernel_time(dig_ctx* ctx, double* total_ms, int64_t* launches) {
  if (!ctx || !total_ms || !launches) return DIG_ERR_ARG;
  int rc = wait_stream(ctx);
  if (rc) return rc;
  double tot = 0.0;
  for (size_t i = 0; i + 1 < ctx->tev_used; i += 2) {
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, ctx->tev[i], ctx->tev[i + 1]));
    tot += ms;
  }
  *total_ms = tot;
  *launches = (int64_t)(ctx->tev_used / 2);
  ctx->tev_used = 0;
  return DIG_OK;
}

// ---------------------------------------------------------------------------
// checkpoint / resume: the host counters and the whole arena
// ---------------------------------------------------------------------------
namespace {
struct CkptHeader {
  char magic[8];
  int64_t version, n_tets, capacity, arena_bytes, rot_dof;
  double mass, dt, F_N;
  uint64_t seed;
  // host state
  int64_t cur, N, have_particles, step, n_ewma, n_win, n_cum, host_steps, flux_steps, n_couple, cl_set, adam_t,
      tile_cells;
  dig_config cfg;  // the configuration the state was made under (after dig_create's defaults)
};
const char kMagic[8] = {'D', 'I', 'G', 'C', 'K', 'P', 'T', '2'};

// the first field that changes results and differs between two
// configurations (nullptr: none); launch shapes and the host wait limit do not
// change results and are not compared
const char* config_mismatch(const dig_config& a, const dig_config& b) {
#define DIG_CMP(f) \
  if (!(a.f == b.f)) return #f;
  DIG_CMP(mass) DIG_CMP(d_ref) DIG_CMP(omega) DIG_CMP(T_ref) DIG_CMP(alpha) DIG_CMP(Z_rot) DIG_CMP(rot_dof)
  DIG_CMP(max_cross) DIG_CMP(F_N) DIG_CMP(dt) DIG_CMP(seed) DIG_CMP(n_init) DIG_CMP(T_init) DIG_CMP(u_init[0])
  DIG_CMP(u_init[1]) DIG_CMP(u_init[2]) DIG_CMP(mu_ref) DIG_CMP(Kn) DIG_CMP(L_ref) DIG_CMP(n_a) DIG_CMP(N_s)
  DIG_CMP(N_m) DIG_CMP(passes) DIG_CMP(eps_m) DIG_CMP(KnD_max) DIG_CMP(capacity) DIG_CMP(closure) DIG_CMP(recon)
  DIG_CMP(local_acc) DIG_CMP(aa_m) DIG_CMP(cfl)
#undef DIG_CMP
  return nullptr;
}
}  // namespace

int dig_checkpoint_bytes(dig_ctx* ctx, int64_t* bytes) {
  if (!ctx || !bytes) return DIG_ERR_ARG;
  if (!ctx->bound) return fail(ctx, DIG_ERR_STATE, "dig_checkpoint_bytes: no arena bound");
  *bytes = (int64_t)sizeof(CkptHeader) + ctx->arena_bytes;
  return DIG_OK;
}

int dig_save(dig_ctx* ctx, void* host_out, int64_t cap) {
  if (!ctx || !host_out) return DIG_ERR_ARG;
  if (!ctx->bound) return fail(ctx, DIG_ERR_STATE, "dig_save: no arena bound");
  if (cap < (int64_t)sizeof(CkptHeader) + ctx->arena_bytes) return fail(ctx, DIG_ERR_CAPACITY, "dig_save: buffer too small");
  CkptHeader h{};
  std::memcpy(h.magic, kMagic, 8);
  h.version = 2;
  h.n_tets = ctx->n_tets;
  h.capacity = ctx->cfg.capacity;
  h.arena_bytes = ctx->arena_bytes;
  h.rot_dof = ctx->cfg.rot_dof;
  h.mass = ctx->cfg.mass;
  h.dt = ctx->cfg.dt;
  h.F_N = ctx->cfg.F_N;
  h.seed = ctx->cfg.seed;
  h.cur = ctx->cur;
  h.N = ctx->N;
  h.have_particles = ctx->have_particles;
  h.step = ctx->step;
  h.n_ewma = ctx->n_ewma;
  h.n_win = ctx->n_win;
  h.n_cum = ctx->n_cum;
  h.host_steps = ctx->host_steps;
  h.flux_steps = ctx->flux_steps;
  h.n_couple = ctx->n_couple;
  h.cl_set = ctx->cl_set;
  h.adam_t = ctx->adam_t;
  h.tile_cells = ctx->tile_cells;
  h.cfg = ctx->cfg;
  int rc = wait_stream(ctx);
  if (rc) return rc;
  std::memcpy(host_out, &h, sizeof h);
  CK(cudaMemcpyAsync((char*)host_out + sizeof h, ctx->arena, (size_t)ctx->arena_bytes, cudaMemcpyDeviceToHost,
                     ctx->stream));
  return wait_stream(ctx);
}

int dig_load(dig_ctx* ctx, const void* host_in, int64_t size) {
  if (!ctx || !host_in) return DIG_ERR_ARG;
  if (!ctx->bound) return fail(ctx, DIG_ERR_STATE, "dig_load: no arena bound");
  if (size < (int64_t)sizeof(CkptHeader)) return fail(ctx, DIG_ERR_ARG, "dig_load: not a checkpoint");
  CkptHeader h;
  std::memcpy(&h, host_in, sizeof h);
  if (std::memcmp(h.magic, kMagic, 8) != 0 || h.version != 2) return fail(ctx, DIG_ERR_ARG, "dig_load: not a checkpoint");
  if (h.n_tets != ctx->n_tets || h.capacity != ctx->cfg.capacity || h.arena_bytes != ctx->arena_bytes ||
      h.rot_dof != ctx->cfg.rot_dof || h.mass != ctx->cfg.mass || h.dt != ctx->cfg.dt || h.F_N != ctx->cfg.F_N ||
      h.seed != ctx->cfg.seed)
    return fail(ctx, DIG_ERR_STATE, "dig_load: checkpoint of a different configuration or mesh");
  if (const char* f = config_mismatch(h.cfg, ctx->cfg)) {
    char msg[160];
    std::snprintf(msg, sizeof msg, "dig_load: checkpoint made with a different dig_config.%s", f);
    return fail(ctx, DIG_ERR_STATE, msg);
  }
  if (size < (int64_t)sizeof h + h.arena_bytes) return fail(ctx, DIG_ERR_ARG, "dig_load: truncated checkpoint");
  int rc = wait_stream(ctx);
  if (rc) return rc;
  CK(cudaMemcpyAsync(ctx->arena, (const char*)host_in + sizeof h, (size_t)h.arena_bytes, cudaMemcpyHostToDevice,
                     ctx->stream));
  rc = wait_stream(ctx);
  if (rc) return rc;
  ctx->cur = (int)h.cur;
  ctx->N = h.N;
  ctx->have_particles = h.have_particles != 0;
  ctx->step = h.step;
  ctx->n_ewma = h.n_ewma;
  ctx->n_win = h.n_win;
  ctx->n_cum = h.n_cum;
  ctx->host_steps = h.host_steps;
  ctx->flux_steps = h.flux_steps;
  ctx->n_couple = h.n_couple;
  ctx->cl_set = h.cl_set != 0;
  if (ctx->have_particles) choose_tile(ctx);  // tiles sized for the restored particle count
  ctx->adam_t = h.adam_t;
  ctx->tile_cells = (int)h.tile_cells;
  return DIG_OK;
}

// ---------------------------------------------------------------------------
// DIG coupling (Alg. 1, one outer step)
// ---------------------------------------------------------------------------
// The synthetic solve (S10) runs in chunks of S10_CHUNK iterations.  A chunk's
// launches have arguments fixed once the arena is bound (pointers,
// configuration, mesh constants; the iteration index and the stopping state
// live on the device), so it is captured once, on a private stream, into a
// CUDA graph and replayed on the context's stream until the solve reports
// itself done (converged, N_m reached or a non-finite residual); the kernels
// of a chunk that runs past that point return at once.  If the capture is
// refused, the kernels are launched directly.
static constexpr int S10_CHUNK = 25;

static int run_s10(dig_ctx* ctx) {
  cudaStream_t s = ctx->stream;
  CK(cudaGetLastError());  // a launch error of the steps before, reported before any capture
  if (!ctx->s10_exec) {
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess) {
      cudaGraph_t gr = nullptr;
      if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        ctx->s10_launches = launch_couple_s10_iters(ctx->P, ctx->C, S10_CHUNK, cs);
        if (cudaStreamEndCapture(cs, &gr) == cudaSuccess && gr) {
          if (cudaGraphInstantiate(&ctx->s10_exec, gr, 0) != cudaSuccess) ctx->s10_exec = nullptr;
          cudaGraphDestroy(gr);
        }
      }
      cudaStreamDestroy(cs);
    }
    (void)cudaGetLastError();  // a refused capture leaves its error here
  }
  launch_couple_s10_init(ctx->P, ctx->C, s);
  const int chunks = (ctx->cfg.N_m + S10_CHUNK - 1) / S10_CHUNK + 1;  // + 1: the chunk that finds N_m reached
  for (int k = 0; k < chunks; ++k) {
    if (ctx->s10_exec) {
      CK(cudaGraphLaunch(ctx->s10_exec, s));
      g_launches += ctx->s10_launches;
    } else {
      g_launches += launch_couple_s10_iters(ctx->P, ctx->C, S10_CHUNK, s);
    }
    int done = 0;
    CK(cudaMemcpyAsync(&done, &ctx->C.scal->done, sizeof(int), cudaMemcpyDeviceToHost, s));
    int rc = wait_stream(ctx);
    if (rc) return rc;
    if (done) break;
  }
  launch_couple_s10_final(ctx->P, ctx->C, s);
  return DIG_OK;
}

int dig_couple(dig_ctx* ctx, dig_couple_report* out) {
  if (!ctx || !out) return DIG_ERR_ARG;
  if (!ctx->have_particles) return fail(ctx, DIG_ERR_STATE, "dig_couple: no particles");
  if (ctx->cfg.N_m < 0 || ctx->cfg.passes < 0) return fail(ctx, DIG_ERR_ARG, "dig_couple: bad N_m or passes");
  std::memset(out, 0, sizeof *out);
  cudaStream_t s = ctx->stream;
  CoupleParams& C = ctx->C;
  C.wall_t = ctx->flux_steps > 0 ? (double)ctx->flux_steps * ctx->cfg.dt : 0.0;
  C.acc_w0 = (double)std::min<int64_t>(ctx->n_ewma, ctx->cfg.n_a);
  CK(cudaMemsetAsync(C.stats, 0, 5 * sizeof(unsigned long long), s));
  CK(cudaMemsetAsync(C.fillcnt, 0, DIG_FILL_LAYERS * sizeof(int), s));
  CK(cudaMemsetAsync(C.scal, 0, sizeof(CoupleScalars), s));
  CK(cudaMemsetAsync(C.clone_total, 0, sizeof(int), s));
  const bool learned = ctx->cfg.closure == 1 && ctx->cl_set;
  if (learned) {
    // S12: the closure's inputs from the coupling window, then its outputs
    launch_closure_features(ctx->P, C, ctx->P.phi_win, (double)ctx->n_win, C.feat, s);
    CK(cudaMemsetAsync(ctx->fw_status, 0, sizeof(int), s));
    launch_mlp_forward(ctx->cl_p, C.feat, ctx->n_tets, C.ypred, ctx->fw_status, s);
    int rf = check_forward(ctx);
    if (rf) return rf;
  }
  int* av = nullptr;
  launch_couple_s9(ctx->P, C, ctx->cfg.passes, learned ? C.ypred : nullptr, &av, s);
  // further chunks of fill layers while the last layer of a chunk still filled cells
  for (int q = DIG_FILL_CHUNK; q < DIG_FILL_LAYERS; q += DIG_FILL_CHUNK) {
    int last = 0;
    CK(cudaMemcpyAsync(&last, C.fillcnt + q - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    int rw = wait_stream(ctx);
    if (rw) return rw;
    if (last == 0) break;
    launch_couple_fill(ctx->P, C, q, q + DIG_FILL_CHUNK, &av, s);
  }
  launch_couple_unreached(ctx->P, C, av, s);
  int rs = run_s10(ctx);
  if (rs) return rs;
  CoupleScalars sc{};
  int N = 0;
  CK(cudaMemcpyAsync(&sc, C.scal, sizeof sc, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&N, ctx->P.cs + ctx->n_tets, sizeof(int), cudaMemcpyDeviceToHost, s));
  int rc = wait_stream(ctx);
  if (rc) return rc;
  out->iters = sc.iters;
  // the result is the best iterate when the last one is worse (k_cp_final)
  const double res = sc.res <= sc.res_best ? sc.res : sc.res_best;
  out->residual = res / (sc.res0 > 0 ? sc.res0 : 1.0);
  const uint32_t sub = (uint32_t)ctx->n_couple;
  ctx->n_couple++;
  bool solved = !sc.bad && std::isfinite(res);
  if (solved) {
    launch_couple_s11(ctx->P, C, ctx->buf[ctx->cur], N, sub, ctx->P.aq, s);
    launch_scan(ctx->P, s);
    launch_scatter(ctx->P, ctx->buf[ctx->cur].mc, s);
    pass(ctx, 0, 0, 0, 0, 0.0, 1.0);
  }
  CK(cudaMemsetAsync(ctx->P.bflux, 0, 5 * std::max<size_t>(ctx->bf.size(), 1) * sizeof(double), s));
  ctx->flux_steps = 0;
  unsigned long long st[5];
  CK(cudaMemcpyAsync(st, C.stats, sizeof st, cudaMemcpyDeviceToHost, s));
  rc = check_status(ctx);
  out->n_learned = (int32_t)st[4];
  out->n_rejected = (int64_t)st[0];
  out->n_reconstructed = (int64_t)st[1];
  out->n_cloned = (int64_t)st[2];
  out->n_deleted = (int64_t)st[3];
  if (rc) return rc;
  if (!solved) return fail(ctx, DIG_ERR_SOLVE, "synthetic solve failed (non-finite or non-positive state)");
  return DIG_OK;
}

int dig_read_couple(dig_ctx* ctx, int32_t which, double* out, int64_t cap) {
  if (!ctx || !out || which < 0 || which > 5) return DIG_ERR_ARG;
  if (!ctx->bound) return fail(ctx, DIG_ERR_STATE, "dig_read_couple: no arena");
  const CoupleParams& C = ctx->C;
  const double* src = which == 0 ? C.half : which == 1 ? C.hot : which == 2 ? C.newst : which == 3 ? C.flag
                    : which == 4 ? C.own : ctx->P.acc_w;
  const int k = which == 1 ? 12 : which == 3 || which == 5 ? 1 : 6;
  const int64_t n = ctx->n_tets;
  if (cap < k * n) return fail(ctx, DIG_ERR_CAPACITY, "dig_read_couple: buffer too small");
  std::vector<double> tmp((size_t)k * n);
  CK(cudaMemcpyAsync(tmp.data(), src, tmp.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  int rc = wait_stream(ctx);
  if (rc) return rc;
  for (int64_t c = 0; c < n; ++c)
    for (int q = 0; q < k; ++q) out[c * k + q] = tmp[(size_t)q * n + c];
  return DIG_OK;
}

int dig_write_moments(dig_ctx* ctx, int32_t which, const double* in) {
  if (!ctx || !in || which < 0 || which > 3) return DIG_ERR_ARG;
  if (!ctx->bound) return fail(ctx, DIG_ERR_STATE, "dig_write_moments: no arena");
  const int64_t n = ctx->n_tets;
  double* dst = which == DIG_PHI_INST ? ctx->P.phi_inst : which == DIG_PHI_EWMA ? ctx->P.phi_ewma
              : which == DIG_PHI_WINDOW ? ctx->P.phi_win : ctx->P.phi_cum;
  std::vector<double> tmp((size_t)NPHI * n);
  for (int64_t c = 0; c < n; ++c)
    for (int q = 0; q < NPHI; ++q) tmp[(size_t)q * n + c] = in[c * NPHI + q];
  CK(cudaMemcpyAsync(dst, tmp.data(), tmp.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  if (which == DIG_PHI_EWMA && ctx->n_ewma == 0) ctx->n_ewma = 1;
  return wait_stream(ctx);
}

int dig_write_wall_flux(dig_ctx* ctx, const double* in, int64_t steps) {
  if (!ctx || !in || steps < 0) return DIG_ERR_ARG;
  if (!ctx->bound) return fail(ctx, DIG_ERR_STATE, "dig_write_wall_flux: no arena");
  if (!ctx->bf.empty())
    CK(cudaMemcpyAsync(ctx->P.bflux, in, 5 * ctx->bf.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  ctx->flux_steps = steps;
  return wait_stream(ctx);
}

// ---------------------------------------------------------------------------
// standalone bucket sort
// ---------------------------------------------------------------------------
int dig_sort_scratch_bytes(int64_t n, int32_t n_cells, int64_t* bytes) {
  if (!bytes || n < 0 || n > INT32_MAX || n_cells <= 0) return fail0(DIG_ERR_ARG, "dig_sort_scratch_bytes: bad sizes");
  *bytes = (int64_t)sort_scratch_bytes(n, n_cells);
  return DIG_OK;
}

int dig_sort_by_cell(const int32_t* cell, int64_t n, int32_t n_cells, int32_t* cell_start, int32_t* order,
                     void* scratch, int64_t scratch_bytes, void* stream) {
  if (n < 0 || n > INT32_MAX || n_cells <= 0 || !cell_start || !scratch || (n > 0 && (!cell || !order)))
    return fail0(DIG_ERR_ARG, "dig_sort_by_cell: bad arguments");
  if (((uintptr_t)scratch & 255) != 0) return fail0(DIG_ERR_ARG, "dig_sort_by_cell: scratch must be 256-byte aligned");
  if (scratch_bytes < (int64_t)sort_scratch_bytes(n, n_cells))
    return fail0(DIG_ERR_CAPACITY, "dig_sort_by_cell: scratch smaller than dig_sort_scratch_bytes()");
  launch_sort_by_cell(cell, n, n_cells, cell_start, order, (char*)scratch, (cudaStream_t)stream);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail0(DIG_ERR_CUDA, cudaGetErrorString(e));
  return DIG_OK;
}

int dig_launch_count(dig_ctx* ctx, int64_t* n) {
  if (!n) return DIG_ERR_ARG;
  *n = (int64_t)g_launches;
  return DIG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// learned closure (S12/S13)
// ---------------------------------------------------------------------------
static int closure_reset_adam(dig_ctx* ctx) {
  cudaStream_t s = ctx->stream;
  CK(cudaMemsetAsync(ctx->cl_m, 0, MLP_NPARAM * sizeof(float), s));
  CK(cudaMemsetAsync(ctx->cl_v, 0, MLP_NPARAM * sizeof(float), s));
  CK(cudaMemsetAsync(ctx->cl_g, 0, MLP_NPARAM * sizeof(float), s));
  ctx->adam_t = 0;
  ctx->cl_set = true;
  return DIG_OK;
}

int closure_init(dig_ctx* ctx, uint64_t seed) {
  if (!ctx) return DIG_ERR_ARG;
  if (!ctx->bound) return fail(ctx, DIG_ERR_STATE, "closure_init: no arena");
  launch_mlp_init(ctx->P, seed, ctx->cl_p, ctx->stream);
  CK(cudaGetLastError());
  return closure_reset_adam(ctx);
}

int closure_set(dig_ctx* ctx, const float* params, int64_t n) {
  if (!ctx || !params) return DIG_ERR_ARG;
  if (n != MLP_NPARAM) return fail(ctx, DIG_ERR_ARG, "closure_set: n must be DIG_MLP_NPARAM");
  if (!ctx->bound) return fail(ctx, DIG_ERR_STATE, "closure_set: no arena");
  CK(cudaMemcpyAsync(ctx->cl_p, params, MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  int rc = closure_reset_adam(ctx);
  if (rc) return rc;
  return wait_stream(ctx);
}

int closure_get(dig_ctx* ctx, float* params, int64_t n) {
  if (!ctx || !params) return DIG_ERR_ARG;
  if (n != MLP_NPARAM) return fail(ctx, DIG_ERR_ARG, "closure_get: n must be DIG_MLP_NPARAM");
  if (!ctx->cl_set) return fail(ctx, DIG_ERR_STATE, "closure_get: no parameters set");
  CK(cudaMemcpyAsync(params, ctx->cl_p, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
  return wait_stream(ctx);
}

static const double* phi_of(dig_ctx* ctx, int which, double* cnt) {
  *cnt = which == DIG_PHI_WINDOW ? (double)ctx->n_win : which == DIG_PHI_CUM ? (double)ctx->n_cum : 1.0;
  return which == DIG_PHI_INST ? ctx->P.phi_inst : which == DIG_PHI_EWMA ? ctx->P.phi_ewma
       : which == DIG_PHI_WINDOW ? ctx->P.phi_win : ctx->P.phi_cum;
}

int closure_features(dig_ctx* ctx, int32_t which, float* X) {
  if (!ctx || !X || which < 0 || which > 3) return DIG_ERR_ARG;
  if (!ctx->bound) return fail(ctx, DIG_ERR_STATE, "closure_features: no arena");
  double cnt;
  const double* phi = phi_of(ctx, which, &cnt);
  launch_closure_features(ctx->P, ctx->C, phi, cnt, X, ctx->stream);
  CK(cudaGetLastError());
  return DIG_OK;
}

int closure_targets(dig_ctx* ctx, int32_t which, const float* X, int64_t n_rows, float* Y) {
  if (!ctx || which < 0 || which > 3 || n_rows < 0 || (n_rows > 0 && (!X || !Y))) return DIG_ERR_ARG;
  if (!ctx->bound) return fail(ctx, DIG_ERR_STATE, "closure_targets: no arena");
  double cnt;
  const double* phi = phi_of(ctx, which, &cnt);
  launch_closure_targets(ctx->P, ctx->C, phi, cnt, X, n_rows, Y, ctx->stream);
  CK(cudaGetLastError());
  return DIG_OK;
}

// the status of the closure's tensor-core forward pass just launched (its
// flag is cleared before every launch); synchronous: DIG_ERR_TIMEOUT if one
// of its waits gave up
static int check_forward(dig_ctx* ctx) {
  int st = 0;
  CK(cudaMemcpyAsync(&st, ctx->fw_status, sizeof st, cudaMemcpyDeviceToHost, ctx->stream));
  int rc = wait_stream(ctx);
  if (rc) return rc;
  if (st) return fail(ctx, DIG_ERR_TIMEOUT, "closure forward: a wait on the tensor cores gave up");
  return DIG_OK;
}

int dig_test_forward_timeout(dig_ctx* ctx) {
  if (!ctx) return DIG_ERR_ARG;
  if (!ctx->bound) return fail(ctx, DIG_ERR_STATE, "dig_test_forward_timeout: no arena bound");
  const long long n = std::min<long long>(128, ctx->n_tets);
  CK(cudaMemsetAsync(ctx->fw_status, 0, sizeof(int), ctx->stream));
  launch_mlp_forward(ctx->cl_p, ctx->C.feat, n, ctx->C.ypred, ctx->fw_status, ctx->stream, 1);
  CK(cudaGetLastError());
  return check_forward(ctx);
}

int closure_forward(dig_ctx* ctx, const float* X, int64_t n, float* Y) {
  if (!ctx || n < 0 || (n > 0 && (!X || !Y))) return DIG_ERR_ARG;
  if (!ctx->cl_set) return fail(ctx, DIG_ERR_STATE, "closure_forward: no parameters set");
  CK(cudaMemsetAsync(ctx->fw_status, 0, sizeof(int), ctx->stream));
  launch_mlp_forward(ctx->cl_p, X, n, Y, ctx->fw_status, ctx->stream);
  CK(cudaGetLastError());
  return check_forward(ctx);
}

int closure_loss(dig_ctx* ctx, const float* X, const float* Y, int64_t n, int32_t identity, double* loss) {
  if (!ctx || !loss || n <= 0 || !X || !Y) return DIG_ERR_ARG;
  if (!identity && !ctx->cl_set) return fail(ctx, DIG_ERR_STATE, "closure_loss: no parameters set");
  cudaStream_t s = ctx->stream;
  CK(cudaMemsetAsync(ctx->cl_acc, 0, 2 * sizeof(double), s));
  CK(cudaMemsetAsync(ctx->fw_status, 0, sizeof(int), s));
  launch_mlp_loss(ctx->cl_p, X, Y, n, identity ? 1 : 0, ctx->cl_acc, ctx->fw_status, s);
  CK(cudaGetLastError());
  double acc = 0.0;
  CK(cudaMemcpyAsync(&acc, ctx->cl_acc, sizeof acc, cudaMemcpyDeviceToHost, s));
  int rc = check_forward(ctx);
  if (rc) return rc;
  *loss = acc / (double)(MLP_NOUT * n);
  return DIG_OK;
}

int closure_grad(dig_ctx* ctx, const float* X, const float* Y, int64_t n, float* grad, double* loss) {
  if (!ctx || !grad || !loss || n <= 0 || !X || !Y) return DIG_ERR_ARG;
  if (!ctx->cl_set) return fail(ctx, DIG_ERR_STATE, "closure_grad: no parameters set");
  cudaStream_t s = ctx->stream;
  CK(cudaMemsetAsync(ctx->cl_g, 0, MLP_NPARAM * sizeof(float), s));
  CK(cudaMemsetAsync(ctx->cl_acc, 0, 2 * sizeof(double), s));
  CK(cudaMemsetAsync(ctx->cl_status, 0, 2 * sizeof(int), s));
  launch_mlp_train_step(ctx->cl_p, X, Y, nullptr, n, 0, n, ctx->cl_g, ctx->cl_acc, ctx->cl_status, s);
  CK(cudaGetLastError());
  double acc = 0.0;
  int st = 0;
  CK(cudaMemcpyAsync(grad, ctx->cl_g, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&acc, ctx->cl_acc, sizeof acc, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&st, ctx->cl_status, sizeof st, cudaMemcpyDeviceToHost, s));
  CK(cudaMemsetAsync(ctx->cl_g, 0, MLP_NPARAM * sizeof(float), s));
  int rc = wait_stream(ctx);
  if (rc) return rc;
  if (st & 2) return fail(ctx, DIG_ERR_TIMEOUT, "closure_grad: a wait on the tensor cores gave up");
  *loss = acc / (double)(MLP_NOUT * n);
  return DIG_OK;
}

int closure_train(dig_ctx* ctx, const dig_train_cfg* cfg, const float* X, const float* Y, int64_t n,
                  double* loss) {
  if (!ctx || !cfg || !loss || n <= 0 || !X || !Y) return DIG_ERR_ARG;
  if (cfg->epochs < 1 || cfg->batch < 1 || !(cfg->lr > 0.0) || !(cfg->beta1 >= 0.0 && cfg->beta1 < 1.0) ||
      !(cfg->beta2 >= 0.0 && cfg->beta2 < 1.0) || !(cfg->eps > 0.0))
    return fail(ctx, DIG_ERR_ARG, "closure_train: bad epochs, batch or Adam constants");
  if (n >= (1LL << 31)) return fail(ctx, DIG_ERR_ARG, "closure_train: n must be < 2^31");
  if (!ctx->cl_set) return fail(ctx, DIG_ERR_STATE, "closure_train: no parameters set");
  cudaStream_t s = ctx->stream;
  CK(cudaMemsetAsync(ctx->cl_status, 0, 2 * sizeof(int), s));
  for (int e = 0; e < cfg->epochs; ++e) {
    CK(cudaMemsetAsync(ctx->cl_acc, 0, 2 * sizeof(double), s));
    const int32_t* perm = cfg->perm ? cfg->perm + (size_t)e * (size_t)n : nullptr;
    for (int64_t b0 = 0; b0 < n; b0 += cfg->batch) {
      const int64_t nb = std::min<int64_t>(cfg->batch, n - b0);
      launch_mlp_train_step(ctx->cl_p, X, Y, perm, n, b0, nb, ctx->cl_g, ctx->cl_acc, ctx->cl_status, s);
      launch_adam(ctx->cl_p, ctx->cl_m, ctx->cl_v, ctx->cl_g, ++ctx->adam_t, (float)cfg->lr, (float)cfg->beta1,
                  (float)cfg->beta2, (float)cfg->eps, s);
    }
    CK(cudaGetLastError());
    double acc = 0.0;
    int st = 0;
    CK(cudaMemcpyAsync(&acc, ctx->cl_acc, sizeof acc, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&st, ctx->cl_status, sizeof st, cudaMemcpyDeviceToHost, s));
    int rc = wait_stream(ctx);
    if (rc) return rc;
    if (st & 2) return fail(ctx, DIG_ERR_TIMEOUT, "closure_train: a wait on the tensor cores gave up");
    if (st) return fail(ctx, DIG_ERR_ARG, "closure_train: a perm entry is outside [0, n)");
    loss[e] = acc / (double)(MLP_NOUT * n);
  }
  return DIG_OK;
}
