// dig_kernels.cu -- sm_103a kernels of the DSMC particle loop.
//
// Compiled with -fmad=false: every floating-point expression is evaluated as
// written (no contraction), and explicit __fma_rn is used where the method
// states a fused multiply-add.  Together with the IEEE-rounded division and
// square root and the FP32 ln/exp below (built from +,-,*,/ only), every
// decision the particle loop takes (cell of a particle, pair indices,
// acceptance, wall re-emission) is a fixed sequence of IEEE operations.
//
// Step structure on the GPU (paper Sec. 2.1: move, then collide pairs of the
// same cell, then sample; Sec. 4 keeps per-cell particle buckets).  The
// particles of cell c occupy slots [cs[c], cs[c+1]) of a buffer in the
// canonical order: stayers of the last move in their previous order, then
// arrivals in the order of their previous slot.
//   k_order      warp per cell: the canonical order (stayers by ballot over
//                the cell's old slot range, arrivals ranked by slot), written
//                as the slot map src (output slot -> input slot), and the
//                velocities (and I_r) gathered into the output buffer.
//   k_collide    thread per cell over the whole mesh: the cell's NTC loop on
//                its gathered velocities.  Every cell's serial candidate
//                chain runs at once, so their latencies overlap.
//   k_move       CTA per tile of cells: the cells' summation variables, then
//                every particle's move x + v dt with the FP32-proven inside
//                test, a proven one-crossing shortcut, and a queue of the rest.
//                A particle's position is one 24-byte record (x, y, z) and
//                its velocity one 12-byte record, so gathering either through
//                the slot map touches one or two sectors.
//   k_track      face-by-face tracking of the queued particles, thread per
//                particle: the dependent mesh loads and FP64 tests of the
//                crossings (FP64 issues at 1/64 of the FP32 rate here)
//                overlap across many warps.
//   k_scan_*     exclusive scans of (stayers + arrivals) and arrivals per cell.
//   k_scatter    appends each mover to its destination cell's arrival list.
// The counting sort of the particle loop therefore costs one 4-byte read of
// the destination cells plus the arrival lists of the movers.
#include "dig_internal.h"
#include "dig_philox.cuh"

#include <cmath>
#include <cstdio>

namespace dig {

std::atomic<long long> g_launches{0};

__device__ __forceinline__ void rng(const Params& P, uint32_t purpose, uint32_t ent, uint32_t sub,
                                    uint32_t step, uint32_t draw, uint32_t (&w)[4]) {
  philox(ent, sub, step, draw, P.seed_lo, P.seed_hi ^ (purpose << 24), w);
}

// FP32 ln: exponent split plus 2 atanh(s), s = (m-1)/(m+1), series to s^11.
__device__ __forceinline__ float ln_f(float x) {
  const uint32_t b = __float_as_uint(x);
  int e = (int)((b >> 23) & 0xffu) - 127;
  if (e == -127) return -87.3365448f;
  float m = __uint_as_float((b & 0x7fffffu) | 0x3f800000u);
  if (m > 1.41421356f) {
    m = m * 0.5f;
    e = e + 1;
  }
  const float s = (m - 1.0f) / (m + 1.0f);
  const float z = s * s;
  float p = 0.0909090909f;
  p = p * z + 0.111111111f;
  p = p * z + 0.142857143f;
  p = p * z + 0.2f;
  p = p * z + 0.333333333f;
  p = p * z + 1.0f;
  const float lnm = (2.0f * s) * p;
  const float fe = (float)e;
  return fe * 0.693145751953125f + (lnm + fe * 1.42860677e-6f);
}

// FP32 exp: 2^k exp(r), Taylor series of exp(r) to r^7, ln 2 split in two parts.
__device__ __forceinline__ float exp_f(float y) {
  if (y < -87.0f) return 0.0f;
  if (y > 88.0f) y = 88.0f;
  const float t = y * 1.44269504f;
  const int k = (int)(t >= 0.0f ? t + 0.5f : t - 0.5f);
  const float fk = (float)k;
  const float r = (y - fk * 0.693145751953125f) - fk * 1.42860677e-6f;
  float p = 1.98412698e-4f;
  p = p * r + 1.38888889e-3f;
  p = p * r + 8.33333333e-3f;
  p = p * r + 4.16666667e-2f;
  p = p * r + 0.166666667f;
  p = p * r + 0.5f;
  p = p * r + 1.0f;
  p = p * r + 1.0f;
  return p * __uint_as_float((uint32_t)(k + 127) << 23);
}

__device__ __forceinline__ float pow_f(float x, float a) { return exp_f(a * ln_f(x)); }

// Exact FP32 -> FP64 conversion with integer operations only, every input
// (zero, subnormal, infinite and NaN included): keeps the FP64 pipe, which
// issues at 1/64 of the FP32 rate, free for arithmetic.
__device__ __forceinline__ double f2d(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned s = b & 0x80000000u;
  const unsigned e = (b >> 23) & 0xffu;
  const unsigned m = b & 0x7fffffu;
  unsigned hi, lo;
  if (e != 0u && e != 255u) {
    hi = s | ((e + 896u) << 20) | (m >> 3);
    lo = m << 29;
  } else if (e == 255u) {
    hi = s | 0x7ff00000u | (m >> 3);
    lo = m << 29;
  } else if (m == 0u) {
    hi = s;
    lo = 0u;
  } else {
    // subnormal m 2^-149: leading one at bit p, exponent p - 149
    const int p = 31 - __clz((int)m);
    const unsigned fr = (m << (23 - p)) & 0x7fffffu;
    hi = s | ((unsigned)(p + 874) << 20) | (fr >> 3);
    lo = fr << 29;
  }
  return __hiloint2double((int)hi, (int)lo);
}

// Gaussian pair, Marsaglia's polar method; two attempts per Philox block;
// returns the index of the first unused draw.
__device__ uint32_t gauss2_next(const Params& P, uint32_t purpose, uint32_t ent, uint32_t sub, uint32_t step,
                                uint32_t draw0, float& g1, float& g2) {
  for (uint32_t d = draw0; d < draw0 + 32; ++d) {
    uint32_t w[4];
    rng(P, purpose, ent, sub, step, d, w);
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const float u1 = 2.0f * u01f(w[2 * a]) - 1.0f;
      const float u2 = 2.0f * u01f(w[2 * a + 1]) - 1.0f;
      const float s = u1 * u1 + u2 * u2;
      if (s < 1.0f && s > 0.0f) {
        const float f = sqrtf(-2.0f * ln_f(s) / s);
        g1 = u1 * f;
        g2 = u2 * f;
        return d + 1;
      }
    }
  }
  g1 = 0.0f;
  g2 = 0.0f;
  return draw0 + 32;
}

// Gaussian pair, Marsaglia's polar method; two attempts per Philox block.
__device__ void gauss2(const Params& P, uint32_t purpose, uint32_t ent, uint32_t sub, uint32_t step,
                       uint32_t draw0, float& g1, float& g2) {
  for (uint32_t d = draw0; d < draw0 + 32; ++d) {
    uint32_t w[4];
    rng(P, purpose, ent, sub, step, d, w);
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const float u1 = 2.0f * u01f(w[2 * a]) - 1.0f;
      const float u2 = 2.0f * u01f(w[2 * a + 1]) - 1.0f;
      const float s = u1 * u1 + u2 * u2;
      if (s < 1.0f && s > 0.0f) {
        const float f = sqrtf(-2.0f * ln_f(s) / s);
        g1 = u1 * f;
        g2 = u2 * f;
        return;
      }
    }
  }
  g1 = 0.0f;
  g2 = 0.0f;
}

// isotropic unit vector (Marsaglia 1972): (a, b) uniform in the unit disc,
// e = (2a sqrt(1-s), 2b sqrt(1-s), 1-2s), s = a^2 + b^2
// isotropic unit vector with the words of the first draw already at hand;
// further draws (rare: both attempts of the first draw rejected) follow
__device__ __forceinline__ void unit_vec_from(const Params& P, const uint32_t (&w0)[4], uint32_t ent, uint32_t sub,
                                              uint32_t step, float& ex, float& ey, float& ez) {
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const float a1 = 2.0f * u01f(w0[2 * a]) - 1.0f;
    const float b1 = 2.0f * u01f(w0[2 * a + 1]) - 1.0f;
    const float s = a1 * a1 + b1 * b1;
    if (s < 1.0f) {
      const float r = 2.0f * sqrtf(1.0f - s);
      ex = a1 * r;
      ey = b1 * r;
      ez = 1.0f - 2.0f * s;
      return;
    }
  }
  for (uint32_t d = 1; d < 32; ++d) {
    uint32_t w[4];
    rng(P, RP_DIR, ent, sub, step, d, w);
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const float a1 = 2.0f * u01f(w[2 * a]) - 1.0f;
      const float b1 = 2.0f * u01f(w[2 * a + 1]) - 1.0f;
      const float s = a1 * a1 + b1 * b1;
      if (s < 1.0f) {
        const float r = 2.0f * sqrtf(1.0f - s);
        ex = a1 * r;
        ey = b1 * r;
        ez = 1.0f - 2.0f * s;
        return;
      }
    }
  }
  ex = 0.0f;
  ey = 0.0f;
  ez = 1.0f;
}

// Post-collision direction of the relative velocity under the VSS model
// (paper Sec. 2.1; Koura & Matsumoto 1991).  The impact parameter obeys
// b/d = cos^alpha(chi/2) with (b/d)^2 uniform, so cos chi = 2 R^(1/alpha) - 1
// for R uniform in (0,1); the azimuth about u = g/|g| is uniform, its cosine
// and sine taken from a uniform point (a, b) of the unit disc as
// (a^2 - b^2)/s and 2ab/s, s = a^2 + b^2.  The direction is
// cos chi u + sin chi (sin eps A + cos eps B) with the orthonormal pair
// A = (q, -u_x u_y/q, -u_x u_z/q), B = (0, u_z/q, -u_y/q), q = |(u_y, u_z)|,
// or A = (0, 1, 0), B = (0, 0, 1) when q <= 1e-6 (g along x).  Random words:
// w0 (draw 0) gives R (word 0) and the first disc point (words 1, 2); draws
// 1..31 two points each (words 0,1 and 2,3).  g2 = |g|^2 > 0.
__device__ __forceinline__ void vss_dir_from(const Params& P, const uint32_t (&w0)[4], uint32_t ent, uint32_t sub,
                                             uint32_t step, float gx, float gy, float gz, float g2, float& ex,
                                             float& ey, float& ez) {
  const float ct = 2.0f * pow_f(u01f(w0[0]), P.inv_alpha) - 1.0f;
  const float st = sqrtf((1.0f - ct) * (1.0f + ct));
  float ce = 1.0f, se = 0.0f;
  bool found = false;
  {
    const float a1 = 2.0f * u01f(w0[1]) - 1.0f;
    const float b1 = 2.0f * u01f(w0[2]) - 1.0f;
    const float s = a1 * a1 + b1 * b1;
    if (s < 1.0f && s > 0.0f) {
      ce = (a1 * a1 - b1 * b1) / s;
      se = 2.0f * a1 * b1 / s;
      found = true;
    }
  }
  for (uint32_t d = 1; d < 32 && !found; ++d) {
    uint32_t w[4];
    rng(P, RP_DIR, ent, sub, step, d, w);
    for (int k0 = 0; k0 <= 2 && !found; k0 += 2) {
      const float a1 = 2.0f * u01f(w[k0]) - 1.0f;
      const float b1 = 2.0f * u01f(w[k0 + 1]) - 1.0f;
      const float s = a1 * a1 + b1 * b1;
      if (s < 1.0f && s > 0.0f) {
        ce = (a1 * a1 - b1 * b1) / s;
        se = 2.0f * a1 * b1 / s;
        found = true;
      }
    }
  }
  const float gn = sqrtf(g2);
  const float ux = gx / gn, uy = gy / gn, uz = gz / gn;
  const float qn = sqrtf(uy * uy + uz * uz);
  if (qn > 1e-6f) {
    ex = ct * ux + st * se * qn;
    ey = ct * uy + st * (ce * uz - se * ux * uy) / qn;
    ez = ct * uz - st * (ce * uy + se * ux * uz) / qn;
  } else {
    ex = ct * ux;
    ey = ct * uy + st * se;
    ez = ct * uz + st * ce;
  }
}

struct Cnt {
  unsigned cand = 0, coll = 0, lb = 0, cross = 0, wall = 0, removed = 0, stuck = 0;
};

// ---------------------------------------------------------------------------
// wall interaction (diffuse at T_w with wall velocity, or specular)
// ---------------------------------------------------------------------------
template <bool DIAT>
__device__ void wall_reflect(const Params& P, int ib, float& vx, float& vy, float& vz, float& I, uint32_t slot,
                             uint32_t hit, uint32_t step, bool flux) {
  const BFaceDev B = P.bf[ib];
  const BCDev bc = P.bc[B.bc];
  const float ix = vx, iy = vy, iz = vz, iI = I;
  if (bc.kind == 1) {
    const float vn = vx * B.nrm[0] + vy * B.nrm[1] + vz * B.nrm[2];
    const float h = 2.0f * vn;
    vx = vx - h * B.nrm[0];
    vy = vy - h * B.nrm[1];
    vz = vz - h * B.nrm[2];
  } else {
    uint32_t w[4];
    rng(P, RP_WALL, slot, hit, step, 0, w);
    const float sg = bc.sigma;
    const float vn = sg * sqrtf(-2.0f * ln_f(u01f(w[0])));
    float g1, g2;
    gauss2(P, RP_WALL, slot, hit, step, 1, g1, g2);
    const float a = sg * g1, b = sg * g2;
    vx = ((bc.U[0] + B.t1[0] * a) + B.t2[0] * b) - B.nrm[0] * vn;
    vy = ((bc.U[1] + B.t1[1] * a) + B.t2[1] * b) - B.nrm[1] * vn;
    vz = ((bc.U[2] + B.t1[2] * a) + B.t2[2] * b) - B.nrm[2] * vn;
    if (DIAT) I = -bc.T * ln_f(u01f(w[1]));
  }
  if (flux) {
    double* F = P.bflux + 5 * (size_t)ib;
    const double m = P.mass_fn;
    atomicAdd(F + 0, 1.0);
    atomicAdd(F + 1, m * ((double)ix - (double)vx));
    atomicAdd(F + 2, m * ((double)iy - (double)vy));
    atomicAdd(F + 3, m * ((double)iz - (double)vz));
    const double ein = (double)ix * ix + (double)iy * iy + (double)iz * iz;
    const double eout = (double)vx * vx + (double)vy * vy + (double)vz * vz;
    atomicAdd(F + 4, 0.5 * m * (ein - eout) + P.fn_kb * ((double)iI - (double)I));
  }
}

__device__ __forceinline__ double dot3(const Plane64& n, double x, double y, double z) {
  return __fma_rn(n.nz, z, __fma_rn(n.ny, y, __dmul_rn(n.nx, x)));
}

// FP64 -> FP32 by truncation with integer operations only (no FP64 pipe):
// |result - x| <= 2^-23 |x|; values below 2^-126 in magnitude become 0.
__device__ __forceinline__ float d2f_trunc(double x) {
  const int hi = __double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const int e = (hi >> 20) & 0x7ff;
  const unsigned m = ((unsigned)(hi & 0xfffff) << 3) | (lo >> 29);
  const unsigned s = (unsigned)hi & 0x80000000u;
  return e > 896 ? __uint_as_float(s | ((unsigned)(e - 896) << 23) | m) : 0.0f;
}

// FP32 plane test d - n.x of a truncated position.  Its error against the
// exact value is below P.margin / 4 (see the margin in dig_api.cu), so
// s > margin proves that the FP64 test d - n.x >= 0 passes and s < -margin
// proves that it fails.
__device__ __forceinline__ float plane_test32(const float4 q, float fx, float fy, float fz) {
  return q.w - __fmaf_rn(q.z, fz, __fmaf_rn(q.y, fy, q.x * fx));
}

// Exit face of the step's ray from `cell`, decided as the FP64 rule decides it:
//   among faces f != entry with b_f = n_f.v > 0, the smallest hit time
//   a_f / b_f with a_f = max(0, d_f - n_f.o) (o: the ray origin), comparing
//   f before g iff a_f b_g < a_g b_f (ties: lowest f); the face is crossed
//   within the step iff !(a_f >= t_rem b_f).
// FP32 interval estimates of b_f and of the hit times decide both answers
// when they separate them; otherwise everything is evaluated in FP64 exactly
// as stated.  Returns the face (-1: none) and sets *cross.
struct Exit {
  int face;
  bool cross;
};

__device__ __forceinline__ Exit exit_face_fp64(const Plane64* pl, int entry, double ox, double oy, double oz,
                                               double vdx, double vdy, double vdz, double trem) {
  int best = -1;
  double ab = 0.0, bb = 1.0;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    if (f == entry) continue;
    const Plane64 q = pl[f];
    const double b = dot3(q, vdx, vdy, vdz);
    if (!(b > 0.0)) continue;
    double a = __dsub_rn(q.d, dot3(q, ox, oy, oz));
    if (a < 0.0) a = 0.0;
    if (best < 0 || __dmul_rn(a, bb) < __dmul_rn(ab, b)) {
      best = f;
      ab = a;
      bb = b;
    }
  }
  Exit r;
  r.face = best;
  r.cross = best >= 0 && !(ab >= __dmul_rn(trem, bb));
  return r;
}

__device__ __forceinline__ Exit exit_face(const Params& P, const Plane64* pl, const float4* pf, int entry,
                                          double ox, double oy, double oz, float fox, float foy, float foz,
                                          double vdx, double vdy, double vdz, float vx, float vy, float vz,
                                          double trem) {
  const float eb = 8.0f * 5.9604645e-08f * (fabsf(vx) + fabsf(vy) + fabsf(vz)) + 1e-30f;
  const float ea = 0.5f * P.margin;
  float lo[4], hi[4];
  bool cand[4];
  bool decided = true;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    cand[f] = false;
    lo[f] = 0.0f;
    hi[f] = 0.0f;
    if (f == entry) continue;
    const float4 q = pf[f];
    const float b = __fmaf_rn(q.z, vz, __fmaf_rn(q.y, vy, q.x * vx));
    if (b < -eb) continue;
    if (!(b > eb)) {
      decided = false;
      continue;
    }
    cand[f] = true;
    const float a = plane_test32(q, fox, foy, foz);
    const float al = fmaxf(a - ea, 0.0f), ah = fmaxf(a + ea, 0.0f);
    const float tl = __fdividef(al, b + eb), th = __fdividef(ah, b - eb);
    lo[f] = tl - tl * 9.5367432e-07f;
    hi[f] = th + th * 9.5367432e-07f + 1e-30f;
  }
  Exit r;
  r.face = -1;
  r.cross = false;
  if (decided) {
    float H = 0.0f;
#pragma unroll
    for (int f = 0; f < 4; ++f)
      if (cand[f] && (r.face < 0 || hi[f] < H)) {
        r.face = f;
        H = hi[f];
      }
#pragma unroll
    for (int f = 0; f < 4; ++f)
      if (cand[f] && f != r.face && !(lo[f] > H)) decided = false;
    if (decided && r.face >= 0) {
      const float T = (float)trem;
      if (H < T * 0.99999f)
        r.cross = true;
      else if (lo[r.face] > T * 1.00001f)
        r.cross = false;
      else
        decided = false;
    }
  }
  if (decided) return r;
  return exit_face_fp64(pl, entry, ox, oy, oz, vdx, vdy, vdz, trem);
}

// Face-by-face tracking of one particle for one time step (the same rule as
// the oracle): ray from o = x to e = o + v t_rem; while e is outside the
// current cell, cross the exit face (exit_face); at a wall the hit time
// a_f / b_f is computed in FP64, o moves to the hit point, the particle is
// re-emitted and e is recomputed.  Returns the final cell or -1 when the
// particle leaves through an open boundary.  FP32 tests only shortcut
// decisions they prove (plane_test32, exit_face).
template <bool DIAT>
__device__ int track(const Params& P, double& x, double& y, double& z, float& vx, float& vy, float& vz, float& I,
                     int cell, uint32_t slot, uint32_t step, bool flux, Cnt& cnt, double trem, int entry) {
  uint32_t hits = 0;
  double ox = x, oy = y, oz = z;
  double vdx = f2d(vx), vdy = f2d(vy), vdz = f2d(vz);
  double ex = __fma_rn(vdx, trem, ox), ey = __fma_rn(vdy, trem, oy), ez = __fma_rn(vdz, trem, oz);
  float fox = d2f_trunc(ox), foy = d2f_trunc(oy), foz = d2f_trunc(oz);
  float fex = d2f_trunc(ex), fey = d2f_trunc(ey), fez = d2f_trunc(ez);
  for (int ncross = 0;; ++ncross) {
    if (ncross > P.max_cross) {
      cnt.stuck++;
      x = ox;
      y = oy;
      z = oz;
      return cell;
    }
    const Plane64* pl = P.plane + 4 * (size_t)cell;
    const float4* pf = P.plane32 + 4 * (size_t)cell;
    bool all_in = true, some_out = false;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      if (f == entry) continue;
      const float s = plane_test32(pf[f], fex, fey, fez);
      if (!(s > P.margin)) all_in = false;
      if (s < -P.margin) some_out = true;
    }
    bool inside = all_in;
    if (!all_in && !some_out) {
      inside = true;
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        if (f == entry) continue;
        const Plane64 q = pl[f];
        if (__dsub_rn(q.d, dot3(q, ex, ey, ez)) < 0.0) inside = false;
      }
    }
    if (inside) {
      x = ex;
      y = ey;
      z = ez;
      return cell;
    }
    const Exit X = exit_face(P, pl, pf, entry, ox, oy, oz, fox, foy, foz, vdx, vdy, vdz, vx, vy, vz, trem);
    if (!X.cross) {
      x = ex;
      y = ey;
      z = ez;
      return cell;
    }
    const int best = X.face;
    cnt.cross++;
    const int nb = __ldg(P.nbr + 4 * (size_t)cell + best);
    if (nb >= 0) {
      entry = __ldg(P.nbrf + 4 * (size_t)cell + best);
      cell = nb;
      continue;
    }
    const int ib = -1 - nb;
    const int kind = P.bc[P.bf[ib].bc].kind;
    if (kind <= 1) {
      const Plane64 q = pl[best];
      const double b = dot3(q, vdx, vdy, vdz);
      double a = __dsub_rn(q.d, dot3(q, ox, oy, oz));
      if (a < 0.0) a = 0.0;
      const double th = __ddiv_rn(a, b);
      ox = __fma_rn(vdx, th, ox);
      oy = __fma_rn(vdy, th, oy);
      oz = __fma_rn(vdz, th, oz);
      trem = __dsub_rn(trem, th);
      wall_reflect<DIAT>(P, ib, vx, vy, vz, I, slot, hits, step, flux);
      hits++;
      cnt.wall++;
      vdx = f2d(vx);
      vdy = f2d(vy);
      vdz = f2d(vz);
      ex = __fma_rn(vdx, trem, ox);
      ey = __fma_rn(vdy, trem, oy);
      ez = __fma_rn(vdz, trem, oz);
      fox = d2f_trunc(ox);
      foy = d2f_trunc(oy);
      foz = d2f_trunc(oz);
      fex = d2f_trunc(ex);
      fey = d2f_trunc(ey);
      fez = d2f_trunc(ez);
      entry = best;
      continue;
    }
    cnt.removed++;
    return -1;
  }
}

// ---------------------------------------------------------------------------
// NTC collisions of one cell (Bird 1994 Sec. 11.1), VHS cross sections with
// isotropic (VHS) or VSS scattering, serial Borgnakke-Larsen exchange (paper
// Eq. inelastic_probability).  Candidates are processed in order k = 0, 1, ...
// on the cell's velocities in the gathered buffer.
// ---------------------------------------------------------------------------
template <bool DIAT, bool VSS>
__device__ void collide_cell(const Params& P, int cell, float* v, float* I, int N, uint32_t step, bool record,
                             Cnt& cnt) {
  if (N < 2) return;
  // the cell's velocity records: particle k's components at v[3k], v[3k+1], v[3k+2]
  auto vx = [v](int k) -> float& { return v[3 * k]; };
  auto vy = [v](int k) -> float& { return v[3 * k + 1]; };
  auto vz = [v](int k) -> float& { return v[3 * k + 2]; };
  float cmax = P.cmax[cell];
  const double X = (double)N * (double)(N - 1) * 0.5 * (double)cmax * P.fdtv[cell] + P.rem[cell];
  const double fl = floor(X);
  P.rem[cell] = X - fl;
  const long long ncand = (long long)fl;
  long long pbase = 0;
  if (record) pbase = (long long)atomicAdd(P.pair_count, (unsigned long long)ncand);
  uint32_t w[4];
  if (ncand > 0) rng(P, RP_COLL, (uint32_t)cell, 0u, step, 0, w);
  for (long long k = 0; k < ncand; ++k) {
    // random words of the next candidate and of this candidate's first
    // direction draw: independent of this candidate's arithmetic, so they
    // overlap with its dependent FP32 chain
    uint32_t wn[4], wd[4];
    if (k + 1 < ncand) rng(P, RP_COLL, (uint32_t)cell, (uint32_t)(k + 1), step, 0, wn);
    rng(P, RP_DIR, (uint32_t)cell, (uint32_t)k, step, 0, wd);
    const int i = (int)(((unsigned long long)w[0] * (unsigned long long)N) >> 32);
    int j = (int)(((unsigned long long)w[1] * (unsigned long long)(N - 1)) >> 32);
    if (j >= i) j = j + 1;
    const float gx = vx(i) - vx(j), gy = vy(i) - vy(j), gz = vz(i) - vz(j);
    float g2 = gx * gx + gy * gy + gz * gz;
    const float g2_pre = g2;
    const float sc = g2 > 0.0f ? P.c_vhs * pow_f(g2, P.one_m_omega) : 0.0f;
    if (sc > cmax) cmax = sc;
    const float R = u01f(w[2]);
    const bool acc = sc > R * cmax;
    cnt.cand++;
    if (record && pbase + k < P.pair_cap) {
      int* r = P.pairs + 4 * (pbase + k);
      r[0] = cell;
      r[1] = (int)k;
      r[2] = i;
      r[3] = j;
      P.pacc[pbase + k] = acc ? 1 : 0;
    }
    if (!acc) {
#pragma unroll
      for (int q = 0; q < 4; ++q) w[q] = wn[q];
      continue;
    }
    cnt.coll++;
    if (DIAT) {
      uint32_t u[4];
      rng(P, RP_LB, (uint32_t)cell, (uint32_t)k, step, 0, u);
      float Etr = g2 * P.hmr;
      if (u01f(u[0]) < P.p_inel) {
        const float Ec = Etr + I[i];
        const float In = Ec * (1.0f - pow_f(u01f(u[1]), P.lb_exp));
        I[i] = In;
        Etr = Ec - In;
        cnt.lb++;
      }
      if (u01f(u[2]) < P.p_inel) {
        const float Ec = Etr + I[j];
        const float In = Ec * (1.0f - pow_f(u01f(u[3]), P.lb_exp));
        I[j] = In;
        Etr = Ec - In;
        cnt.lb++;
      }
      g2 = Etr / P.hmr;
    }
    const float cr = sqrtf(g2);
    float ex, ey, ez;
    if (VSS)
      vss_dir_from(P, wd, (uint32_t)cell, (uint32_t)k, step, gx, gy, gz, g2_pre, ex, ey, ez);
    else
      unit_vec_from(P, wd, (uint32_t)cell, (uint32_t)k, step, ex, ey, ez);
#pragma unroll
    for (int q = 0; q < 4; ++q) w[q] = wn[q];
    const float h = 0.5f * cr;
    float cm;
    cm = (vx(i) + vx(j)) * 0.5f;
    vx(i) = cm + h * ex;
    vx(j) = cm - h * ex;
    cm = (vy(i) + vy(j)) * 0.5f;
    vy(i) = cm + h * ey;
    vy(j) = cm - h * ey;
    cm = (vz(i) + vz(j)) * 0.5f;
    vz(i) = cm + h * ez;
    vz(j) = cm - h * ez;
  }
  P.cmax[cell] = cmax;
}

// per-cell summation variables of one cell, one warp: FP32 partial sums per
// lane (strided over the cell's particles), then a reduce-scatter across the
// warp (16 shuffles instead of one full reduction per component).  Returns
// in lanes 2q and 2q+1 the cell's sum of component q + 1 (components 1..16:
// v(3), vv (xx,yy,zz,xy,xz,yz), |v|^2 v(3), I, I v(3); 13..16 zero for a
// monatomic gas).
template <bool DIAT>
__device__ __forceinline__ float cell_sums_warp(const float* v, const float* I, int N, int lane) {
  float s[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) s[q] = 0.0f;
  for (int k = lane; k < N; k += 32) {
    const float x = v[3 * k], y = v[3 * k + 1], z = v[3 * k + 2];
    const float vv = x * x + y * y + z * z;
    s[0] += x;
    s[1] += y;
    s[2] += z;
    s[3] += x * x;
    s[4] += y * y;
    s[5] += z * z;
    s[6] += x * y;
    s[7] += x * z;
    s[8] += y * z;
    s[9] += vv * x;
    s[10] += vv * y;
    s[11] += vv * z;
    if (DIAT) {
      const float e = I[k];
      s[12] += e;
      s[13] += e * x;
      s[14] += e * y;
      s[15] += e * z;
    }
  }
  // stage o: lanes with bit o set keep the upper half of their values, the
  // others the lower half, each adding its partner's copy of what it keeps
#pragma unroll
  for (int st = 0; st < 4; ++st) {
    const int o = 16 >> st, m = 8 >> st;
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < m; ++i) {
      const float send = up ? s[i] : s[i + m];
      const float keep = up ? s[i + m] : s[i];
      s[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return s[0] + __shfl_xor_sync(0xffffffffu, s[0], 1);
}

__device__ __forceinline__ void flush_counters(const Params& P, const Cnt& c) {
  unsigned v[7] = {c.cand, c.coll, c.lb, c.cross, c.wall, c.removed, c.stuck};
#pragma unroll
  for (int q = 0; q < 7; ++q)
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  if ((threadIdx.x & 31) == 0) {
    const int idx[7] = {C_CAND, C_COLL, C_LB, C_CROSS, C_WALL, C_REMOVED, C_STUCK};
#pragma unroll
    for (int q = 0; q < 7; ++q)
      if (v[q]) atomicAdd(P.counters + idx[q], (unsigned long long)v[q]);
  }
}

// ---------------------------------------------------------------------------
// the particle pass: k_order, k_collide, k_move
// ---------------------------------------------------------------------------

// Canonical order of every cell, half a warp per cell: the two cells of a
// warp proceed together, so their dependent loads overlap (grid-stride over
// cell pairs).  The stayers of cell c are the slots of its old range
// [sbase, sbase + nold) of the input buffer whose mc is c (the move that
// wrote them left them in c), in slot order; the arrivals are the aq entries
// of c (slots of particles that moved into c, new particles included),
// ranked by slot.  Writes src[cs[c] + k], keeps it in shared memory for cells
// of up to OQ particles, gathers velocities (and I_r) into the output buffer
// and records the new range as the cell's old range for the next pass.
constexpr int OQ = 64;

template <bool DIAT>
__global__ void __launch_bounds__(256) k_order(Params P, Buf IN, Buf OUT) {
  __shared__ int s_src[256 / 16][OQ];
  const int lane = threadIdx.x & 31, g = lane >> 4, gl = lane & 15;
  int* my = s_src[threadIdx.x >> 4];
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    P.state[1] = 0;
    P.state[2] = 0;
  }
  const unsigned glt = (1u << gl) - 1u;
  const int npair = (P.n_cells + 1) >> 1;
  for (int pr = gw; pr < npair; pr += nw) {
    const int c = 2 * pr + g;
    const bool live = c < P.n_cells;
    // every independent load of the cell first
    int base = 0, Nc = 0, sb = 0, no = 0, a0 = 0, na = 0;
    if (live) {
      base = P.cs[c];
      Nc = P.cs[c + 1] - base;
      sb = P.sbase[c];
      no = P.nold[c];
      a0 = P.as[c];
      na = P.as[c + 1] - a0;
    }
    const int key = gl < na ? P.aq[a0 + gl] : 0x7fffffff;
    // stayers: 16 old slots per round and cell; the bounds are warp-uniform
    const int no_max = max(no, __shfl_xor_sync(0xffffffffu, no, 16));
    // the old slots' cells are loaded four rounds ahead of their ballots, and
    // the gathered velocities four rounds ahead of their stores, so that the
    // loads of a cell overlap
    int ns = 0;
    for (int k1 = 0; k1 < no_max; k1 += 64) {
      int mv[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int k = k1 + 16 * r + gl;
        mv[r] = k < no ? IN.mc[sb + k] : -2;
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int k0 = k1 + 16 * r;
        if (k0 >= no_max) break;
        const int k = k0 + gl;
        const bool st = k < no && mv[r] == c;
        const unsigned bs = (__ballot_sync(0xffffffffu, st) >> (16 * g)) & 0xffffu;
        const int pos = ns + __popc(bs & glt);
        if (st && pos < Nc) {
          P.src[base + pos] = sb + k;
          if (pos < OQ) my[pos] = sb + k;
        }
        ns += __popc(bs);
      }
    }
    // arrivals, ranked by slot
    const int na_max = max(na, __shfl_xor_sync(0xffffffffu, na, 16));
    if (na_max <= 16) {
      int rank = 0;
      for (int r = 0; r < na_max; ++r) {
        const int kr = __shfl_sync(0xffffffffu, key, 16 * g + r);
        rank += (r < na && kr < key) ? 1 : 0;
      }
      const int pos = ns + rank;
      if (gl < na && pos < Nc) {
        P.src[base + pos] = key;
        if (pos < OQ) my[pos] = key;
      }
    } else {
      for (int r = gl; r < na; r += 16) {
        const int kk = P.aq[a0 + r];
        int rank = 0;
        for (int r2 = 0; r2 < na; ++r2) rank += (P.aq[a0 + r2] < kk) ? 1 : 0;
        const int pos = ns + rank;
        if (pos < Nc) {
          P.src[base + pos] = kk;
          if (pos < OQ) my[pos] = kk;
        }
      }
    }
    __syncwarp();
    for (int k1 = gl; k1 < Nc; k1 += 64) {
      float ax[4], ay[4], az[4], ai[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int k = k1 + 16 * r;
        if (k < Nc) {
          const int q = k < OQ ? my[k] : P.src[base + k];
          ax[r] = IN.vel[3 * (size_t)q];
          ay[r] = IN.vel[3 * (size_t)q + 1];
          az[r] = IN.vel[3 * (size_t)q + 2];
          if (DIAT) ai[r] = IN.Ir[q];
        }
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int k = k1 + 16 * r;
        if (k < Nc) {
          float* vo = OUT.vel + 3 * (size_t)(base + k);
          vo[0] = ax[r];
          vo[1] = ay[r];
          vo[2] = az[r];
          OUT.mc[base + k] = c;  // the slot's cell until k_move writes the destination
          if (DIAT) OUT.Ir[base + k] = ai[r];
        }
      }
    }
    if (live && gl == 0) {
      P.sbase[c] = base;
      P.nold[c] = Nc;
    }
    __syncwarp();
  }
}

// NTC collisions of every cell, thread per cell, on the gathered velocities
template <bool DIAT, bool VSS>
__global__ void __launch_bounds__(128) k_collide(Params P, Buf OUT, uint32_t step, int record) {
  Cnt cnt;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < P.n_cells) {
    const int base = P.cs[c], N = P.cs[c + 1] - base;
    collide_cell<DIAT, VSS>(P, c, OUT.vel + 3 * (size_t)base, DIAT ? OUT.Ir + base : nullptr, N, step, record != 0,
                            cnt);
  }
  flush_counters(P, cnt);
}

// Sampling and move of a tile of TC cells.  Sampling: the FP32 sums of each
// cell (warp per cell) into shared memory, then the FP64 accumulators with
// coalesced accesses, thread per (component, cell).  Move: every particle of
// the tile (its slots are contiguous): x' = x + v dt and the FP32 plane tests
// of x' against its cell (plane_test32).  All four passed with the margin: it
// stays.  Exactly one failed with the margin, the others passed and the
// particle approaches that face: the segment x -> x' leaves through it (a
// convex cell: the only half-space x' violates is the one the segment
// crossed, and the margins order the FP64 hit times the same way), so if the
// face is interior and x' passes the neighbour's other three tests, the
// particle ends there after one crossing -- the result of the full tracking
// rule.  Everything else (walls, several crossings, tests within the margin)
// is queued (output slot, input slot) for k_track, its cell left in mc.
template <bool DIAT, int NT>
__global__ void __launch_bounds__(NT) k_move(Params P, Buf IN, Buf OUT, int pass, int sflags, uint32_t step,
                                             double ewa, double ewb, int TC) {
  extern __shared__ __align__(16) int smem_i[];
  double* s_ea = (double*)smem_i;          // TC moving-average weights of old value
  double* s_eb = s_ea + TC;                // and of the new sample
  int* s_cs = (int*)(s_eb + TC);           // TC + 1 slot starts
  int* s_nst = s_cs + TC + 1;              // TC stayers
  float* s_sum = (float*)(s_nst + TC);     // NPHI x TC cell sums
  const int c0 = blockIdx.x * TC;
  if (c0 >= P.n_cells) return;
  const int nc = min(TC, P.n_cells - c0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = NT / 32;
  // cells in the local accumulation state (Sec. 3.2) take the running mean:
  // weights (w-1)/w and 1/w with w = acc_w + 1, acc_w counting the step
  const bool accw = P.local_acc && (pass & PASS_COLLIDE) && (sflags & S_EWMA);
  for (int i = threadIdx.x; i <= nc; i += NT) {
    s_cs[i] = P.cs[c0 + i];
    if (i < nc) {
      s_nst[i] = 0;
      if (accw) {
        double a = ewa, b = ewb;
        const double aw = P.acc_w[c0 + i];
        if (aw > 0.0) {
          const double w = aw + 1.0;
          P.acc_w[c0 + i] = w;
          a = (w - 1.0) / w;
          b = 1.0 / w;
        }
        s_ea[i] = a;
        s_eb[i] = b;
      }
    }
  }
  __syncthreads();
  Cnt cnt;
  if (pass & PASS_COLLIDE) {
    constexpr int np = DIAT ? 17 : 13;
    for (int c = warp; c < nc; c += nwarps) {
      const int b = s_cs[c], N = s_cs[c + 1] - b;
      const float t = cell_sums_warp<DIAT>(OUT.vel + 3 * (size_t)b, DIAT ? OUT.Ir + b : nullptr, N, lane);
      const int q = (lane >> 1) + 1;
      if ((lane & 1) == 0 && q < np) s_sum[q * nc + c] = t;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < np * nc; i += NT) {
      const int q = i / nc, lc = i - q * nc;
      const size_t o = (size_t)q * (size_t)P.n_cells + (size_t)(c0 + lc);
      const double ph = f2d(q == 0 ? (float)(s_cs[lc + 1] - s_cs[lc]) : s_sum[i]);
      if (sflags & S_INST) P.phi_inst[o] = ph;
      if (sflags & S_EWMA)
        P.phi_ewma[o] = accw ? __fma_rn(s_ea[lc], P.phi_ewma[o], s_eb[lc] * ph) : __fma_rn(ewa, P.phi_ewma[o], ewb * ph);
      if (sflags & S_WINDOW) P.phi_win[o] += ph;
      if (sflags & S_CUMUL) P.phi_cum[o] += ph;
    }
  }
  const bool do_move = (pass & PASS_MOVE) != 0;
  const int lo = s_cs[0], hi = s_cs[nc];
  // loop bounds are warp-uniform: the ballots below see every lane
  for (int b0 = lo + warp * 32; b0 < hi; b0 += NT) {
    const int slot = b0 + lane;
    const bool valid = slot < hi;
    int lc = -1, st = -1, nb = -1;
    if (valid) {
      const int cell = OUT.mc[slot];  // the slot's cell, written by k_order
      lc = cell - c0;
      const int q = P.src[slot];
      const double* pq = IN.pos + 3 * (size_t)q;
      double x = pq[0], y = pq[1], z = pq[2];
      st = 0;
      if (do_move) {
        const float* vs = OUT.vel + 3 * (size_t)slot;
        const float vx = vs[0], vy = vs[1], vz = vs[2];
        x = __fma_rn(f2d(vx), P.dt, x);
        y = __fma_rn(f2d(vy), P.dt, y);
        z = __fma_rn(f2d(vz), P.dt, z);
        const float4* pf = P.plane32 + 4 * (size_t)cell;
        const float fx = d2f_trunc(x), fy = d2f_trunc(y), fz = d2f_trunc(z);
        int nok = 0, nout = 0, fo = 0;
        float4 qo = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          const float4 pq = pf[f];
          const float t = plane_test32(pq, fx, fy, fz);
          if (t > P.margin) {
            ++nok;
          } else if (t < -P.margin) {
            ++nout;
            fo = f;
            qo = pq;
          }
        }
        if (nok != 4) {
          st = 2;
          // the crossed face must also be approached: n.v > 0 proven in FP32
          const float bo = __fmaf_rn(qo.z, vz, __fmaf_rn(qo.y, vy, qo.x * vx));
          const float eb = 8.0f * 5.9604645e-08f * (fabsf(vx) + fabsf(vy) + fabsf(vz)) + 1e-30f;
          if (nout == 1 && nok == 3 && bo > eb) {
            nb = __ldg(P.nbr + 4 * (size_t)cell + fo);
            if (nb >= 0) {
              const int en = __ldg(P.nbrf + 4 * (size_t)cell + fo);
              const float4* pn = P.plane32 + 4 * (size_t)nb;
              bool in = true;
#pragma unroll
              for (int f = 0; f < 4; ++f)
                if (f != en && !(plane_test32(pn[f], fx, fy, fz) > P.margin)) in = false;
              if (in) st = 1;
            }
          }
        }
      }
      if (st <= 1) {
        double* po = OUT.pos + 3 * (size_t)slot;
        po[0] = x;
        po[1] = y;
        po[2] = z;
      }
      OUT.mc[slot] = st == 1 ? nb : cell;
      if (st == 1) {
        atomicAdd(P.na + nb, 1);
        cnt.cross++;
      }
      if (st == 2) lc = -1;
    }
    const bool queued = st == 2;
    const unsigned qm = __ballot_sync(0xffffffffu, queued);
    if (qm) {
      const int leader = __ffs(qm) - 1;
      int qbase = 0;
      if (lane == leader) qbase = atomicAdd(P.state + 3, __popc(qm));
      qbase = __shfl_sync(0xffffffffu, qbase, leader);
      if (queued)
        reinterpret_cast<int2*>(P.tq)[qbase + __popc(qm & ((1u << lane) - 1u))] = make_int2(slot, P.src[slot]);
    }
    const bool stay = st == 0;
    if (__ballot_sync(0xffffffffu, stay)) {
      const unsigned peers = __match_any_sync(0xffffffffu, stay ? lc : 256 + lane);
      if (stay && lane == __ffs(peers) - 1) atomicAdd(s_nst + lc, __popc(peers));
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < nc; c += NT) P.nst[c0 + c] = s_nst[c];
  flush_counters(P, cnt);
}

size_t move_smem(int TC) {
  return sizeof(double) * 2 * (size_t)TC + sizeof(int) * (size_t)(2 * TC + 1) + sizeof(float) * (size_t)NPHI * TC;
}

// ---------------------------------------------------------------------------
// face-by-face tracking of the particles the cell pass queued (those whose
// fast move it could not prove inside their cell): thread per queued
// particle over the whole domain, so the dependent loads and FP64 tests of
// the crossings overlap across many warps.  The cell pass left each one's
// post-collision velocity and its cell at the output slot; the position is
// still the input slot's.  Stayers and arrivals are counted for the sort.
// ---------------------------------------------------------------------------
template <bool DIAT>
__global__ void __launch_bounds__(128) k_track(Params P, Buf IN, Buf OUT, uint32_t step, int flux) {
  const int nq = P.state[3];
  Cnt cnt;
  const int2* tq = reinterpret_cast<const int2*>(P.tq);
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    const int2 e = tq[q];
    const int slot = e.x, src = e.y;
    const int cell = OUT.mc[slot];
    const double* ps = IN.pos + 3 * (size_t)src;
    double x = ps[0], y = ps[1], z = ps[2];
    const float* vs = OUT.vel + 3 * (size_t)slot;
    float vx = vs[0], vy = vs[1], vz = vs[2], I = DIAT ? OUT.Ir[slot] : 0.0f;
    const int dst = track<DIAT>(P, x, y, z, vx, vy, vz, I, cell, (uint32_t)slot, step, flux, cnt, P.dt, -1);
    OUT.pos[3 * (size_t)slot] = x;
    OUT.pos[3 * (size_t)slot + 1] = y;
    OUT.pos[3 * (size_t)slot + 2] = z;
    OUT.vel[3 * (size_t)slot] = vx;
    OUT.vel[3 * (size_t)slot + 1] = vy;
    OUT.vel[3 * (size_t)slot + 2] = vz;
    if (DIAT) OUT.Ir[slot] = I;
    OUT.mc[slot] = dst;
    if (dst == cell)
      atomicAdd(P.nst + cell, 1);
    else if (dst >= 0)
      atomicAdd(P.na + dst, 1);
  }
  flush_counters(P, cnt);
}

// ---------------------------------------------------------------------------
// S4: free-stream injection through inflow faces (Bird's one-sided flux, the
// count carried as an FP64 remainder per face; the normal speed drawn from the
// drifting flux law z exp(-(z-s)^2), z = beta v_n > 0, by acceptance-rejection:
//   s <= 0: z = sqrt(-ln R), accepted with exp(2 s z);
//   s > 0:  dominating function (z-s)^+ e^{-(z-s)^2} + s e^{-(z-s)^2}, masses
//           1/2 and s sqrt(pi): z = s + sqrt(-ln R), or z = s + N(0,1/2)
//           (Gaussian drawn to completion) rejected for z <= 0 and accepted
//           with z/s below s.
// New particles are appended after every existing slot, face-major in
// boundary-face order, then move for a uniform fraction of dt.
// ---------------------------------------------------------------------------
__global__ void k_inj_count(Params P) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P.n_in) return;
  const double X = P.inflow[j].expn + P.inj_rem[j];
  const double fl = floor(X);
  P.inj_rem[j] = X - fl;
  P.inj_cnt[j] = fl > 0.0 ? (int)fl : 0;  // a rounding-negative expectation injects nothing
}

// single-CTA exclusive scan of the per-face counts (inflow faces are few
// compared with particles; the loop walks them in chunks of the block)
__global__ void __launch_bounds__(1024) k_inj_scan(Params P) {
  __shared__ int sh[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int base = 0; base < P.n_in; base += 1024) {
    const int j = base + threadIdx.x;
    const int v = j < P.n_in ? P.inj_cnt[j] : 0;
    int inc = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) sh[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      int w = sh[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      sh[lane] = w;
    }
    __syncthreads();
    const int excl = carry + inc - v + (warp > 0 ? sh[warp - 1] : 0);
    if (j < P.n_in) P.inj_off[j] = excl;
    __syncthreads();
    if (threadIdx.x == 1023) carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    P.inj_off[P.n_in] = carry;
    const int N0 = P.cs[P.n_cells];
    long long hi = (long long)N0 + carry;
    if (hi > P.cap) {
      atomicOr(P.status, ST_CAPACITY);
      hi = P.cap;
    }
    P.state[1] = N0;
    P.state[2] = (int)hi;
  }
}

template <bool DIAT>
__device__ float inflow_normal_speed(const Params& P, const InflowDev& F, uint32_t ib, uint32_t k, uint32_t step,
                                     uint32_t& draw) {
  const float s = F.s;
  for (int att = 0; att < 64; ++att) {
    uint32_t w[4];
    rng(P, RP_INJECT, ib, k, step, draw++, w);
    if (s <= 0.0f) {
      const float z = sqrtf(-ln_f(u01f(w[0])));
      if (u01f(w[1]) < exp_f(2.0f * s * z)) return z;
    } else if (u01f(w[0]) < F.p1) {
      return s + sqrtf(-ln_f(u01f(w[1])));
    } else {
      float g1, g2;
      draw = gauss2_next(P, RP_INJECT, ib, k, step, draw, g1, g2);
      const float z = s + g1 * 0.707106781f;
      if (z > 0.0f && (z >= s || u01f(w[3]) * s < z)) return z;
    }
  }
  return s > 0.0f ? s : 0.5f;
}

template <bool DIAT>
__global__ void k_inj_gen(Params P, Buf OUT, uint32_t step, int wallflux) {
  const int N0 = P.state[1], total = P.state[2] - N0;
  Cnt cnt;
  unsigned inj = 0;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    ++inj;
    // face of this new particle: last j with inj_off[j] <= t
    int lo = 0, hi = P.n_in - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (P.inj_off[mid] <= t)
        lo = mid;
      else
        hi = mid - 1;
    }
    const InflowDev F = P.inflow[lo];
    const uint32_t ib = (uint32_t)F.bface, k = (uint32_t)(t - P.inj_off[lo]);
    const int slot = N0 + t;
    uint32_t w[4];
    rng(P, RP_INJECT, ib, k, step, 0, w);
    double r1 = u01d(w[0], w[1]), r2 = u01d(w[2], w[3]);
    if (r1 + r2 > 1.0) {
      r1 = 1.0 - r1;
      r2 = 1.0 - r2;
    }
    double x = F.a[0] + r1 * (F.b[0] - F.a[0]) + r2 * (F.c[0] - F.a[0]);
    double y = F.a[1] + r1 * (F.b[1] - F.a[1]) + r2 * (F.c[1] - F.a[1]);
    double z = F.a[2] + r1 * (F.b[2] - F.a[2]) + r2 * (F.c[2] - F.a[2]);
    rng(P, RP_INJECT, ib, k, step, 1, w);
    const double tfrac = u01d(w[0], w[1]);
    float g1, g2;
    uint32_t draw = gauss2_next(P, RP_INJECT, ib, k, step, 2, g1, g2);
    const float vn = inflow_normal_speed<DIAT>(P, F, ib, k, step, draw) * F.invb;
    const BFaceDev B = P.bf[F.bface];
    const float a = F.ut1 + F.sig * g1, b = F.ut2 + F.sig * g2;
    float vx = (B.t1[0] * a + B.t2[0] * b) - B.nrm[0] * vn;
    float vy = (B.t1[1] * a + B.t2[1] * b) - B.nrm[1] * vn;
    float vz = (B.t1[2] * a + B.t2[2] * b) - B.nrm[2] * vn;
    float I = 0.0f;
    if (DIAT) {
      rng(P, RP_INJECT, ib, k, step, draw, w);
      I = -P.bc[B.bc].T * ln_f(u01f(w[0]));
    }
    const int dst = track<DIAT>(P, x, y, z, vx, vy, vz, I, F.tet, (uint32_t)slot, step, wallflux != 0, cnt,
                                tfrac * P.dt, F.face);
    OUT.pos[3 * (size_t)slot] = x;
    OUT.pos[3 * (size_t)slot + 1] = y;
    OUT.pos[3 * (size_t)slot + 2] = z;
    OUT.vel[3 * (size_t)slot] = vx;
    OUT.vel[3 * (size_t)slot + 1] = vy;
    OUT.vel[3 * (size_t)slot + 2] = vz;
    if (DIAT) OUT.Ir[slot] = I;
    OUT.mc[slot] = dst;
    if (dst >= 0) atomicAdd(P.na + dst, 1);
  }
  // injected count and the tracking counters of the new particles
  for (int o = 16; o > 0; o >>= 1) inj += __shfl_xor_sync(0xffffffffu, inj, o);
  if ((threadIdx.x & 31) == 0 && inj) atomicAdd(P.counters + C_INJECTED, (unsigned long long)inj);
  flush_counters(P, cnt);
}

// ---------------------------------------------------------------------------
// scans: cs = exclusive scan(nst + na), as = exclusive scan(na); zero na, fill
// ---------------------------------------------------------------------------
constexpr int SCAN_T = 1024, SCAN_ITEMS = 4;
constexpr int SCAN_CHUNK = SCAN_T * SCAN_ITEMS;

int scan_blocks(int n) { return (n + SCAN_CHUNK - 1) / SCAN_CHUNK; }

__global__ void __launch_bounds__(SCAN_T) k_scan_reduce(Params P) {
  const int n = P.n_cells;
  const int base = blockIdx.x * SCAN_CHUNK;
  int tot = 0, arr = 0;
  for (int i = threadIdx.x; i < SCAN_CHUNK; i += SCAN_T) {
    const int c = base + i;
    if (c < n) {
      const int a = P.na[c];
      tot += P.nst[c] + a;
      arr += a;
    }
  }
  __shared__ int sh[2][32];
  for (int o = 16; o > 0; o >>= 1) {
    tot += __shfl_xor_sync(0xffffffffu, tot, o);
    arr += __shfl_xor_sync(0xffffffffu, arr, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = tot;
    sh[1][threadIdx.x >> 5] = arr;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    tot = sh[0][threadIdx.x];
    arr = sh[1][threadIdx.x];
    for (int o = 16; o > 0; o >>= 1) {
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
      arr += __shfl_xor_sync(0xffffffffu, arr, o);
    }
    if (threadIdx.x == 0) {
      P.scan_part[2 * blockIdx.x] = tot;
      P.scan_part[2 * blockIdx.x + 1] = arr;
    }
  }
}

__global__ void __launch_bounds__(SCAN_T) k_scan_final(Params P) {
  const int n = P.n_cells;
  const int base = blockIdx.x * SCAN_CHUNK;
  __shared__ int sh[2][32];
  __shared__ int s_off[2];
  // offset of this block: sum of the partials of the blocks before it
  int pt = 0, pa = 0;
  for (int b = threadIdx.x; b < (int)blockIdx.x; b += SCAN_T) {
    pt += P.scan_part[2 * b];
    pa += P.scan_part[2 * b + 1];
  }
  for (int o = 16; o > 0; o >>= 1) {
    pt += __shfl_xor_sync(0xffffffffu, pt, o);
    pa += __shfl_xor_sync(0xffffffffu, pa, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = pt;
    sh[1][threadIdx.x >> 5] = pa;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int a = 0, b = 0;
    for (int w = 0; w < SCAN_T / 32; ++w) {
      a += sh[0][w];
      b += sh[1][w];
    }
    s_off[0] = a;
    s_off[1] = b;
  }
  __syncthreads();
  // each thread: SCAN_ITEMS consecutive cells
  int vt[SCAN_ITEMS], va[SCAN_ITEMS];
  int lt = 0, la = 0;
  const int c0 = base + threadIdx.x * SCAN_ITEMS;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    const int c = c0 + i;
    int a = 0, t = 0;
    if (c < n) {
      a = P.na[c];
      t = P.nst[c] + a;
    }
    vt[i] = t;
    va[i] = a;
    lt += t;
    la += a;
  }
  // block exclusive scan of (lt, la)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int it = lt, ia = la;
  for (int o = 1; o < 32; o <<= 1) {
    const int yt = __shfl_up_sync(0xffffffffu, it, o), ya = __shfl_up_sync(0xffffffffu, ia, o);
    if (lane >= o) {
      it += yt;
      ia += ya;
    }
  }
  __syncthreads();
  if (lane == 31) {
    sh[0][warp] = it;
    sh[1][warp] = ia;
  }
  __syncthreads();
  if (warp == 0) {
    int wt = sh[0][lane], wa = sh[1][lane];
    for (int o = 1; o < 32; o <<= 1) {
      const int yt = __shfl_up_sync(0xffffffffu, wt, o), ya = __shfl_up_sync(0xffffffffu, wa, o);
      if (lane >= o) {
        wt += yt;
        wa += ya;
      }
    }
    sh[0][lane] = wt;
    sh[1][lane] = wa;
  }
  __syncthreads();
  int et = s_off[0] + it - lt + (warp > 0 ? sh[0][warp - 1] : 0);
  int ea = s_off[1] + ia - la + (warp > 0 ? sh[1][warp - 1] : 0);
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    const int c = c0 + i;
    if (c < n) {
      P.cs[c] = et;
      P.as[c] = ea;
      P.na[c] = 0;
      P.fill[c] = 0;
    }
    et += vt[i];
    ea += va[i];
    if (c == n - 1) {
      P.cs[n] = et;
      P.as[n] = ea;
      P.state[0] = et;
      P.state[3] = 0;  // track queue consumed
      if ((long long)et > P.cap) atomicOr(P.status, ST_CAPACITY);
    }
  }
}

// ---------------------------------------------------------------------------
// scatter movers into their destination cells' arrival lists: a particle at
// slot q of cell c's range moved if mc[q] != c; new particles (initial
// state, host-written, injected) occupy the extra slot range
// ---------------------------------------------------------------------------
__global__ void k_scatter(Params P, const int* __restrict__ mc) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int c = gw; c < P.n_cells; c += nw) {
    const int lo = P.sbase[c], hi = lo + P.nold[c];
    // two rounds of the range per iteration: both cells loaded, both atomics
    // in flight, before the arrival-list stores
    for (int q0 = lo + lane; q0 < hi; q0 += 64) {
      const int q1 = q0 + 32;
      const int d0 = mc[q0];
      const int d1 = q1 < hi ? mc[q1] : c;
      const bool m0 = d0 != c && d0 >= 0 && d0 < P.n_cells;
      const bool m1 = d1 != c && d1 >= 0 && d1 < P.n_cells;
      int a0 = 0, a1 = 0, f0 = 0, f1 = 0;
      if (m0) {
        a0 = P.as[d0];
        f0 = atomicAdd(P.fill + d0, 1);
      }
      if (m1) {
        a1 = P.as[d1];
        f1 = atomicAdd(P.fill + d1, 1);
      }
      if (m0) P.aq[a0 + f0] = q0;
      if (m1) P.aq[a1 + f1] = q1;
    }
  }
  const int lo = P.state[1], hi = P.state[2];
  for (int q = lo + blockIdx.x * blockDim.x + threadIdx.x; q < hi; q += gridDim.x * blockDim.x) {
    const int d = mc[q];
    if (d >= 0 && d < P.n_cells) {
      const int pos = P.as[d] + atomicAdd(P.fill + d, 1);
      P.aq[pos] = q;
    }
  }
}

// ---------------------------------------------------------------------------
// initial state: paper Sec. 5.1 uniform equilibrium; new particles become
// arrivals (keys = their index) of the next cell pass
// ---------------------------------------------------------------------------
template <bool DIAT>
__global__ void k_init(Params P, Buf OUT, int n) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  uint32_t w[4], w2[4];
  const int nt = P.n_cells;
  rng(P, RP_INIT_POS, (uint32_t)p, 0, 0, 0, w);
  const double target = u01d(w[0], w[1]) * P.cumvol[nt - 1];
  int lo = 0, hi = nt - 1;
  while (lo < hi) {
    const int mid = (lo + hi) / 2;
    if (P.cumvol[mid] > target)
      hi = mid;
    else
      lo = mid + 1;
  }
  const int t = lo;
  rng(P, RP_INIT_POS, (uint32_t)p, 1, 0, 0, w);
  rng(P, RP_INIT_POS, (uint32_t)p, 2, 0, 0, w2);
  double s = u01d(w[0], w[1]), tt = u01d(w[2], w[3]), u = u01d(w2[0], w2[1]);
  if (s + tt > 1.0) {
    s = 1.0 - s;
    tt = 1.0 - tt;
  }
  if (tt + u > 1.0) {
    const double tmp = u;
    u = 1.0 - s - tt;
    tt = 1.0 - tmp;
  } else if (s + tt + u > 1.0) {
    const double tmp = u;
    u = s + tt + u - 1.0;
    s = 1.0 - tt - tmp;
  }
  const int* tv = P.tets + 4 * (size_t)t;
  const double* A = P.nodes + 3 * (size_t)tv[0];
  const double* B = P.nodes + 3 * (size_t)tv[1];
  const double* C = P.nodes + 3 * (size_t)tv[2];
  const double* D = P.nodes + 3 * (size_t)tv[3];
  double xs[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) xs[i] = A[i] + s * (B[i] - A[i]) + tt * (C[i] - A[i]) + u * (D[i] - A[i]);
  float g[4];
  gauss2(P, RP_INIT_VEL, (uint32_t)p, 0, 0, 0, g[0], g[1]);
  gauss2(P, RP_INIT_VEL, (uint32_t)p, 1, 0, 0, g[2], g[3]);
  OUT.pos[3 * (size_t)p] = xs[0];
  OUT.pos[3 * (size_t)p + 1] = xs[1];
  OUT.pos[3 * (size_t)p + 2] = xs[2];
  OUT.vel[3 * (size_t)p] = P.u0[0] + P.sigma_init * g[0];
  OUT.vel[3 * (size_t)p + 1] = P.u0[1] + P.sigma_init * g[1];
  OUT.vel[3 * (size_t)p + 2] = P.u0[2] + P.sigma_init * g[2];
  if (DIAT) {
    rng(P, RP_INIT_VEL, (uint32_t)p, 2, 0, 0, w);
    OUT.Ir[p] = -P.T_init * ln_f(u01f(w[0]));
  }
  OUT.mc[p] = t;
  atomicAdd(P.na + t, 1);
}

// host-supplied particles (interleaved staging) -> buffer + arrivals
__global__ void k_write(Params P, Buf OUT, const double* xs, const float* vs, const float* Is, const int* cells,
                        int n, int diat) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  OUT.pos[3 * (size_t)p] = xs[3 * (size_t)p];
  OUT.pos[3 * (size_t)p + 1] = xs[3 * (size_t)p + 1];
  OUT.pos[3 * (size_t)p + 2] = xs[3 * (size_t)p + 2];
  OUT.vel[3 * (size_t)p] = vs[3 * (size_t)p];
  OUT.vel[3 * (size_t)p + 1] = vs[3 * (size_t)p + 1];
  OUT.vel[3 * (size_t)p + 2] = vs[3 * (size_t)p + 2];
  if (diat) OUT.Ir[p] = Is ? Is[p] : 0.0f;
  const int c = cells[p];
  OUT.mc[p] = c;
  atomicAdd(P.na + c, 1);
}

// current sorted buffer -> interleaved staging + cell of each slot
__global__ void k_read(Params P, Buf CUR, double* xs, float* vs, float* Is, int* cells, int n, int diat) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
  for (int p = gt; p < n; p += nt) {
    xs[3 * (size_t)p] = CUR.pos[3 * (size_t)p];
    xs[3 * (size_t)p + 1] = CUR.pos[3 * (size_t)p + 1];
    xs[3 * (size_t)p + 2] = CUR.pos[3 * (size_t)p + 2];
    vs[3 * (size_t)p] = CUR.vel[3 * (size_t)p];
    vs[3 * (size_t)p + 1] = CUR.vel[3 * (size_t)p + 1];
    vs[3 * (size_t)p + 2] = CUR.vel[3 * (size_t)p + 2];
    Is[p] = diat ? CUR.Ir[p] : 0.0f;
  }
  for (int c = gt; c < P.n_cells; c += nt)
    for (int p = P.cs[c]; p < P.cs[c + 1]; ++p) cells[p] = c;
}

// summation variables [NPHI][n] * scale -> [n][NPHI] or derived moments [n][NMAC]
// (paper Eq. dsmc_temperatures from averaged raw sums, SI units)
__global__ void k_moments(Params P, const double* phi, double scale, int macro, double* out, double mass,
                          double FN, double kB) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = P.n_cells;
  if (c >= n) return;
  double ph[NPHI];
#pragma unroll
  for (int q = 0; q < NPHI; ++q) ph[q] = phi[(size_t)q * n + c] * scale;
  if (!macro) {
#pragma unroll
    for (int q = 0; q < NPHI; ++q) out[(size_t)c * NPHI + q] = ph[q];
    return;
  }
  double* M = out + (size_t)c * NMAC;
#pragma unroll
  for (int q = 0; q < NMAC; ++q) M[q] = 0.0;
  const double N = ph[0];
  M[0] = N;
  if (!(N > 0.0)) return;
  const double V = P.vol[c];
  const double u0 = ph[1] / N, u1 = ph[2] / N, u2 = ph[3] / N;
  const double m00 = ph[4] / N, m11 = ph[5] / N, m22 = ph[6] / N, m01 = ph[7] / N, m02 = ph[8] / N,
               m12 = ph[9] / N;
  const double c00 = m00 - u0 * u0, c11 = m11 - u1 * u1, c22 = m22 - u2 * u2;
  const double c01 = m01 - u0 * u1, c02 = m02 - u0 * u2, c12 = m12 - u1 * u2;
  const double tr = c00 + c11 + c22, v2 = m00 + m11 + m22, uu = u0 * u0 + u1 * u1 + u2 * u2;
  const double rho = mass * FN * N / V;
  M[1] = rho;
  M[2] = u0;
  M[3] = u1;
  M[4] = u2;
  const double Tt = mass * tr / (3.0 * kB);
  M[5] = Tt;
  const int dr = P.rot_dof;
  const double Tr = dr > 0 ? 2.0 * (ph[13] / N) / dr : 0.0;
  M[6] = Tr;
  M[7] = (3.0 * Tt + dr * Tr) / (3.0 + dr);
  M[8] = rho * (c00 - tr / 3.0);
  M[9] = rho * (c11 - tr / 3.0);
  M[10] = rho * (c22 - tr / 3.0);
  M[11] = rho * c01;
  M[12] = rho * c02;
  M[13] = rho * c12;
  const double mv[3][3] = {{m00, m01, m02}, {m01, m11, m12}, {m02, m12, m22}};
  const double u[3] = {u0, u1, u2};
  for (int i = 0; i < 3; ++i) {
    const double uj = u[0] * mv[i][0] + u[1] * mv[i][1] + u[2] * mv[i][2];
    const double c3 = ph[10 + i] / N - 2.0 * uj - u[i] * v2 + 2.0 * u[i] * uu;
    M[14 + i] = 0.5 * rho * c3;
    if (dr > 0) M[17 + i] = (FN * N / V) * kB * (ph[14 + i] / N - u[i] * (ph[13] / N));
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static int blocks_for(long long n, int t) { return (int)((n + t - 1) / t); }

void launch_init(const Params& P, const Buf& out, int n, cudaStream_t s) {
  if (n <= 0) return;
  if (P.rot_dof > 0)
    k_init<true><<<blocks_for(n, 256), 256, 0, s>>>(P, out, n);
  else
    k_init<false><<<blocks_for(n, 256), 256, 0, s>>>(P, out, n);
  ++g_launches;
}

void launch_write(const Params& P, const Buf& out, const double* xs, const float* vs, const float* Is,
                  const int* cells, int n, cudaStream_t s) {
  if (n <= 0) return;
  k_write<<<blocks_for(n, 256), 256, 0, s>>>(P, out, xs, vs, Is, cells, n, P.rot_dof > 0);
  ++g_launches;
}

void launch_scan(const Params& P, cudaStream_t s) {
  const int nb = scan_blocks(P.n_cells);
  k_scan_reduce<<<nb, SCAN_T, 0, s>>>(P);
  k_scan_final<<<nb, SCAN_T, 0, s>>>(P);
  g_launches += 2;
}

void launch_scatter(const Params& P, const int* mc, cudaStream_t s) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
  }
  k_scatter<<<sms * 8, 256, 0, s>>>(P, mc);
  ++g_launches;
}

static int sm_count() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
  }
  return sms;
}

template <bool DIAT, int NT>
static void launch_move_t(const Params& P, const Buf& in, const Buf& out, int pass, int sflags, uint32_t step_move,
                          double ewa, double ewb, int TC, cudaStream_t s) {
  const size_t sm = move_smem(TC);
  cudaFuncSetAttribute(k_move<DIAT, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_move<DIAT, NT><<<blocks_for(P.n_cells, TC), NT, sm, s>>>(P, in, out, pass, sflags, step_move, ewa, ewb, TC);
}

// one particle pass: order, collisions (PASS_COLLIDE), sampling and move
// (PASS_MOVE: moving, else the positions are copied), tracking of the queue
void launch_cell_pass(const Params& P, const Buf& in, const Buf& out, int pass, int sflags, uint32_t step_coll,
                      uint32_t step_move, double ewa, double ewb, int TC, int threads, cudaStream_t s) {
  const bool diat = P.rot_dof > 0;
  const int sms = sm_count();
  if (diat)
    k_order<true><<<sms * 16, 256, 0, s>>>(P, in, out);
  else
    k_order<false><<<sms * 16, 256, 0, s>>>(P, in, out);
  g_launches += 1;
  if (pass & PASS_COLLIDE) {
    const int rec = (sflags & S_PAIRS) != 0;
    const int nb = blocks_for(P.n_cells, 128);
    if (diat && P.vss)
      k_collide<true, true><<<nb, 128, 0, s>>>(P, out, step_coll, rec);
    else if (diat)
      k_collide<true, false><<<nb, 128, 0, s>>>(P, out, step_coll, rec);
    else if (P.vss)
      k_collide<false, true><<<nb, 128, 0, s>>>(P, out, step_coll, rec);
    else
      k_collide<false, false><<<nb, 128, 0, s>>>(P, out, step_coll, rec);
    g_launches += 1;
  }
#define DIG_MV(D, T) launch_move_t<D, T>(P, in, out, pass, sflags, step_move, ewa, ewb, TC, s)
  if (threads <= 64) {
    if (diat) DIG_MV(true, 64); else DIG_MV(false, 64);
  } else if (threads <= 128) {
    if (diat) DIG_MV(true, 128); else DIG_MV(false, 128);
  } else {
    if (diat) DIG_MV(true, 256); else DIG_MV(false, 256);
  }
#undef DIG_MV
  g_launches += 1;
  if (pass & PASS_MOVE) {
    const int flux = (sflags & S_WALLFLUX) != 0;
    if (diat)
      k_track<true><<<sms * 16, 128, 0, s>>>(P, in, out, step_move, flux);
    else
      k_track<false><<<sms * 16, 128, 0, s>>>(P, in, out, step_move, flux);
    ++g_launches;
  }
}

void launch_inject(const Params& P, const Buf& out, uint32_t step, int wallflux, cudaStream_t s) {
  if (P.n_in <= 0) return;
  k_inj_count<<<blocks_for(P.n_in, 256), 256, 0, s>>>(P);
  k_inj_scan<<<1, 1024, 0, s>>>(P);
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
  }
  if (P.rot_dof > 0)
    k_inj_gen<true><<<sms * 4, 256, 0, s>>>(P, out, step, wallflux);
  else
    k_inj_gen<false><<<sms * 4, 256, 0, s>>>(P, out, step, wallflux);
  g_launches += 3;
}

namespace {
// He-normal initialisation of the learned closure: weight k of the network
// (layers in order, biases skipped) is the k-th value of the Gaussian pairs
// drawn from the MLP_INIT stream with entity = the pair's first index;
// std sqrt(2 / fan_in) per layer; biases zero
__global__ void k_mlp_init(Params P, float* __restrict__ params, float sd_in, float sd_hid) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;  // pair index
  constexpr int nW[4] = {64 * MLP_NIN, 64 * 64, 64 * 64, MLP_NOUT * 64};
  constexpr int nb[4] = {64, 64, 64, MLP_NOUT};
  const int idx = 2 * k;
  int base = 0, poff = 0, l = 0;
  for (; l < 4; ++l) {
    if (idx < base + nW[l]) break;
    base += nW[l];
    poff += nW[l] + nb[l];
  }
  if (l < 4) {
    float g1, g2;
    gauss2(P, RP_MLP_INIT, (uint32_t)idx, 0, 0, 0, g1, g2);
    const float sd = l == 0 ? sd_in : sd_hid;
    const int i = idx - base;
    params[poff + i] = sd * g1;
    if (i + 1 < nW[l]) params[poff + i + 1] = sd * g2;
  }
  // biases
  if (k < 64 * 3 + MLP_NOUT) {
    int o = 0, j = k;
    for (int q = 0; q < 4; ++q) {
      o += nW[q];
      if (j < nb[q]) {
        params[o + j] = 0.0f;
        break;
      }
      j -= nb[q];
      o += nb[q];
    }
  }
}
}  // namespace

void launch_mlp_init(const Params& P0, uint64_t seed, float* params, cudaStream_t s) {
  Params P = P0;
  P.seed_lo = (uint32_t)seed;
  P.seed_hi = (uint32_t)(seed >> 32);
  const float sd_in = (float)std::sqrt(2.0 / MLP_NIN), sd_hid = (float)std::sqrt(2.0 / 64);
  const int pairs = (64 * MLP_NIN + 2 * 64 * 64 + MLP_NOUT * 64) / 2;
  k_mlp_init<<<(pairs + 255) / 256, 256, 0, s>>>(P, params, sd_in, sd_hid);
  ++g_launches;
}

void launch_read(const Params& P, const Buf& cur, double* xs, float* vs, float* Is, int* cells, int n,
                 cudaStream_t s) {
  k_read<<<256, 256, 0, s>>>(P, cur, xs, vs, Is, cells, n, P.rot_dof > 0);
  ++g_launches;
}

void launch_moments_ex(const Params& P, const double* phi, double scale, int macro, double* out, double mass,
                       double FN, double kB, cudaStream_t s) {
  k_moments<<<blocks_for(P.n_cells, 128), 128, 0, s>>>(P, phi, scale, macro, out, mass, FN, kB);
  ++g_launches;
}

}  // namespace dig
