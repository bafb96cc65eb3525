// dig_couple.cu -- the intermittent DIG coupling on the GPU (paper Sec. 3,
// Alg. 1): S9 HoT extraction with the cell-Knudsen reliability filter and
// layered neighbour reconstruction, S10 the steady synthetic equations, S11
// particle recalibration.  FP64 throughout, one thread per cell (the work is
// per cell and small next to the particle loop).  Multiply-adds may be fused
// here: the fields are compared with the oracle within FP64 tolerances.
//
// Nondimensional variables (Sec. 2.2): lengths / L0, density / (m n0),
// temperature / T0, velocity / sqrt(R T0); p = rho T_t; mu = Kn sqrt(2/pi)
// T_t^omega (the paper's Kn definition); kappa_t = 15/4 mu, kappa_r = 1.32 mu.
// Arrays are component-major, [component][cell].
#include "dig_internal.h"
#include "dig_philox.cuh"

namespace dig {

namespace {

// x^a for normal x > 0 as exp(a ln x), FP64, a few ulp: ln by the exponent
// split and ln m = 2 atanh(s) = 2 s (1 + s^2/3 + s^4/5 + ...), s = (m-1)/(m+1),
// m in [1/sqrt2, sqrt2) (|s| <= 0.1716, series to s^22); exp by Cody-Waite
// reduction y = k ln2 + r, |r| <= ln2/2, and the Taylor series of e^r to r^13.
// ln2 = LN2_HI + LN2_LO with LN2_HI ln2 rounded to 32 significant bits, so that
// k LN2_HI is exact.
__device__ __forceinline__ double pow_pos(double x, double a) {
  constexpr double LN2_HI = 0.6931471803691238, LN2_LO = 1.9082149292705877e-10, INV_LN2 = 1.4426950408889634;
  const long long bits = __double_as_longlong(x);
  int e = (int)((bits >> 52) & 0x7ff) - 1023;
  double m = __longlong_as_double((bits & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
  if (m > 1.4142135623730951) {
    m *= 0.5;
    e += 1;
  }
  const double s = (m - 1.0) / (m + 1.0);
  const double z = s * s;
  double p = 1.0 / 23.0;
  p = fma(p, z, 1.0 / 21.0);
  p = fma(p, z, 1.0 / 19.0);
  p = fma(p, z, 1.0 / 17.0);
  p = fma(p, z, 1.0 / 15.0);
  p = fma(p, z, 1.0 / 13.0);
  p = fma(p, z, 1.0 / 11.0);
  p = fma(p, z, 1.0 / 9.0);
  p = fma(p, z, 1.0 / 7.0);
  p = fma(p, z, 1.0 / 5.0);
  p = fma(p, z, 1.0 / 3.0);
  p = fma(p, z, 1.0);
  const double de = (double)e;
  const double lnx = fma(de, LN2_HI, fma(de, LN2_LO, 2.0 * s * p));
  const double y = a * lnx;
  const double k = rint(y * INV_LN2);
  const double r = fma(-k, LN2_LO, fma(-k, LN2_HI, y));
  double q = 1.0 / 6227020800.0;  // 1/13!
  q = fma(q, r, 1.0 / 479001600.0);
  q = fma(q, r, 1.0 / 39916800.0);
  q = fma(q, r, 1.0 / 3628800.0);
  q = fma(q, r, 1.0 / 362880.0);
  q = fma(q, r, 1.0 / 40320.0);
  q = fma(q, r, 1.0 / 5040.0);
  q = fma(q, r, 1.0 / 720.0);
  q = fma(q, r, 1.0 / 120.0);
  q = fma(q, r, 1.0 / 24.0);
  q = fma(q, r, 1.0 / 6.0);
  q = fma(q, r, 0.5);
  q = fma(q, r, 1.0);
  q = fma(q, r, 1.0);
  return q * __longlong_as_double((long long)((int)k + 1023) << 52);
}

__device__ __forceinline__ double mu_nd(const CoupleParams& C, double Tt) {
  return C.Kn * sqrt(2.0 / M_PI) * pow_pos(Tt > 1e-6 ? Tt : 1e-6, C.omega);
}

// boundary values (walls: wall velocity and temperature; open: free stream)
// values of u (3), T_t and T_r at a boundary face with outward unit normal N,
// seen from a cell with primitives Pc: a diffuse wall or an inflow face gives
// its own velocity and temperature; a specular wall the cell's velocity without
// its normal component and the cell's temperatures (slip, adiabatic); an
// outflow face the cell's own values
__device__ __forceinline__ void bc_values(const Params& P, const CoupleParams& C, int ib, const double* Pc,
                                          const double* N, double* phi) {
  const int b = P.bf[ib].bc;
  const int kind = P.bc[b].kind;
  if (kind == 1) {
    const double un = Pc[1] * N[0] + Pc[2] * N[1] + Pc[3] * N[2];
    for (int i = 0; i < 3; ++i) phi[i] = Pc[1 + i] - un * N[i];
    phi[3] = Pc[4];
    phi[4] = Pc[5];
  } else if (kind == 3) {
    for (int q = 0; q < 5; ++q) phi[q] = Pc[1 + q];
  } else {
    for (int i = 0; i < 3; ++i) phi[i] = C.bcU[3 * b + i] / C.c0;
    phi[3] = C.bcT[b] / C.T0;
    phi[4] = phi[3];
  }
}

// S9: the cell's own state and sampled stress / heat flux from summation
// variables phi summed over cnt steps (cnt = 1: the moving average)
// (Eq. dsmc_temperatures, nondimensional)
__global__ void k_cp_extract(Params P, CoupleParams C, const double* __restrict__ phi, double cnt) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = P.n_cells;
  if (c >= n) return;
  double ph[NPHI];
  for (int q = 0; q < NPHI; ++q) {
    const double v = phi[(size_t)q * n + c];
    ph[q] = cnt == 1.0 ? v : cnt > 0.0 ? v / cnt : 0.0;
  }
  double M[NMAC];
  for (int q = 0; q < NMAC; ++q) M[q] = 0.0;
  const double N = ph[0];
  M[0] = N;
  if (N > 0.0) {
    const double V = P.vol[c];
    const double u0 = ph[1] / N, u1 = ph[2] / N, u2 = ph[3] / N;
    const double m00 = ph[4] / N, m11 = ph[5] / N, m22 = ph[6] / N, m01 = ph[7] / N, m02 = ph[8] / N,
                 m12 = ph[9] / N;
    const double c00 = m00 - u0 * u0, c11 = m11 - u1 * u1, c22 = m22 - u2 * u2;
    const double c01 = m01 - u0 * u1, c02 = m02 - u0 * u2, c12 = m12 - u1 * u2;
    const double tr = c00 + c11 + c22, v2 = m00 + m11 + m22, uu = u0 * u0 + u1 * u1 + u2 * u2;
    const double rho = C.mass * C.FN * N / V;
    M[1] = rho;
    M[2] = u0;
    M[3] = u1;
    M[4] = u2;
    M[5] = C.mass * tr / (3.0 * C.kB);
    M[6] = C.dr > 0 ? 2.0 * (ph[13] / N) / C.dr : 0.0;
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
      if (C.dr > 0) M[17 + i] = (C.FN * N / V) * C.kB * (ph[14 + i] / N - u[i] * (ph[13] / N));
    }
  }
  C.own[0 * (size_t)n + c] = M[1] / C.rho0;
  C.own[1 * (size_t)n + c] = M[2] / C.c0;
  C.own[2 * (size_t)n + c] = M[3] / C.c0;
  C.own[3 * (size_t)n + c] = M[4] / C.c0;
  C.own[4 * (size_t)n + c] = M[5] / C.T0;
  C.own[5 * (size_t)n + c] = C.dr > 0 ? M[6] / C.T0 : M[5] / C.T0;
  const double ss = C.rho0 * C.c0 * C.c0, qs = ss * C.c0;
  for (int q = 0; q < 6; ++q) C.sd[(size_t)q * n + c] = M[8 + q] / ss;
  for (int q = 0; q < 3; ++q) {
    C.sd[(size_t)(6 + q) * n + c] = M[14 + q] / qs;
    C.sd[(size_t)(9 + q) * n + c] = M[17 + q] / qs;
  }
  C.nbar[c] = N;
}

// NSF stress and heat fluxes from the gradients G (du_i/dx_j at 3i+j, then T_t, T_r)
__device__ void nsf_mu(const CoupleParams& C, double mu, const double* G, double* sig, double* qt, double* qr) {
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
    qr[i] = C.dr > 0 ? -kr * G[12 + i] : 0.0;
  }
}

// least-squares gradients of u (3), T_t, T_r of cell c from primitives
// prim[6][n]: grad phi = sum_f w_f (phi_f - phi_c), w_f = M^-1 d_f from the
// mesh tables (neighbour values across interior faces, boundary values at
// boundary faces); exact for linear fields
// (NF = 5 fields; NF = 4 leaves out T_r, whose gradient a monatomic gas does
// not use)
template <int NF = 5>
__device__ __forceinline__ void grad_cell(const Params& P, const CoupleParams& C, const double* __restrict__ prim,
                                          int c, double* g) {
  const int n = P.n_cells;
  double Pc[6];
  for (int q = 0; q < 6; ++q) Pc[q] = prim[(size_t)q * n + c];
  for (int q = 0; q < 15; ++q) g[q] = 0.0;
  for (int f = 0; f < 4; ++f) {
    const int nb = P.nbr[4 * (size_t)c + f];
    double phi[5];
    if (nb >= 0) {
      for (int q = 0; q < NF; ++q) phi[q] = prim[(size_t)(1 + q) * n + nb];
    } else {
      const Plane64 pl = P.plane[4 * (size_t)c + f];
      const double N[3] = {pl.nx, pl.ny, pl.nz};
      bc_values(P, C, -1 - nb, Pc, N, phi);
    }
    const double w0 = C.lsqw[(size_t)(3 * f + 0) * n + c];
    const double w1 = C.lsqw[(size_t)(3 * f + 1) * n + c];
    const double w2 = C.lsqw[(size_t)(3 * f + 2) * n + c];
    for (int q = 0; q < NF; ++q) {
      const double dq = phi[q] - Pc[1 + q];
      g[3 * q + 0] += w0 * dq;
      g[3 * q + 1] += w1 * dq;
      g[3 * q + 2] += w2 * dq;
    }
  }
}

__global__ void k_cp_grad(Params P, CoupleParams C, const double* __restrict__ prim, double* __restrict__ grad) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = P.n_cells;
  if (c >= n) return;
  double g[15];
  grad_cell(P, C, prim, c, g);
  for (int q = 0; q < 15; ++q) grad[(size_t)q * n + c] = g[q];
}

__device__ void nsf(const CoupleParams& C, double Tt, const double* G, double* sig, double* qt, double* qr) {
  nsf_mu(C, mu_nd(C, Tt), G, sig, qt, qr);
}

// HoT = sampled - NSF of cell c (Eq. hot_extraction) from C.own, C.sd, C.grad
__device__ void hot_cell(const Params& P, const CoupleParams& C, int c, double* Pc, double* H) {
  const int n = P.n_cells;
  double G[15];
  for (int q = 0; q < 6; ++q) Pc[q] = C.own[(size_t)q * n + c];
  for (int q = 0; q < 15; ++q) G[q] = C.grad[(size_t)q * n + c];
  double sig[6], qt[3], qr[3];
  nsf(C, Pc[4], G, sig, qt, qr);
  for (int q = 0; q < 6; ++q) H[q] = C.sd[(size_t)q * n + c] - sig[q];
  for (int q = 0; q < 3; ++q) {
    H[6 + q] = C.sd[(size_t)(6 + q) * n + c] - qt[q];
    H[9 + q] = C.sd[(size_t)(9 + q) * n + c] - qr[q];
  }
}

// HoT; cell Knudsen criterion (Eq. criterion); half = own
__global__ void k_cp_hot(Params P, CoupleParams C) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = P.n_cells;
  if (c >= n) return;
  double Pc[6], H[12];
  hot_cell(P, C, c, Pc, H);
  for (int q = 0; q < 12; ++q) C.hot[(size_t)q * n + c] = H[q];
  for (int q = 0; q < 6; ++q) C.half[(size_t)q * n + c] = Pc[q];
  const double V = P.vol[c] / (C.L0 * C.L0 * C.L0);
  const double dc = 2.0 * cbrt(3.0 * V / (4.0 * M_PI));
  // a state needs at least two particles on average to have a temperature
  bool ok = C.nbar[c] >= 2.0 && Pc[0] > 0.0 && Pc[4] > 0.0;
  for (int q = 0; q < 6 && ok; ++q) ok = isfinite(Pc[q]);
  for (int q = 0; q < 12 && ok; ++q) ok = isfinite(H[q]);
  if (ok) {
    const double lam = C.Kn * pow(Pc[4], C.omega - 0.5) / Pc[0];
    ok = lam / dc <= C.KnD_max;
  }
  C.avail[c] = ok ? 1 : 0;
  C.flag[c] = ok ? 1.0 : 0.0;
  if (!ok) atomicAdd(C.stats + 0, 1ull);
  // local accumulation state (Sec. 3.2): a rejected cell stops forgetting, its
  // moving average so far counting as the acc_w0 samples it stands for; an
  // accepted cell returns to the moving average
  if (P.local_acc) {
    if (ok)
      P.acc_w[c] = 0.0;
    else if (P.acc_w[c] == 0.0)
      P.acc_w[c] = C.acc_w0;
  }
}

// S12 inputs of every cell (see closure_features in dig.h): rho, u(3), T_t,
// traceless HoT stress (xx, yy, xy, xz, yz) / (rho T_t), HoT q_t / (rho
// T_t^{3/2}); zero rows for empty cells.  wnorm keeps rho and T_t (0 when
// the row is invalid).
__global__ void k_cl_features(Params P, CoupleParams C, float* __restrict__ X) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = P.n_cells;
  if (c >= n) return;
  double o[6], H[12], f[MLP_NIN];
  hot_cell(P, C, c, o, H);
  bool ok = C.nbar[c] > 0.0 && o[0] > 0.0 && o[4] > 0.0;
  if (ok) {
    const double s = o[0] * o[4], qn = s * sqrt(o[4]);
    f[0] = o[0];
    f[1] = o[1];
    f[2] = o[2];
    f[3] = o[3];
    f[4] = o[4];
    f[5] = H[0] / s;
    f[6] = H[1] / s;
    f[7] = H[3] / s;
    f[8] = H[4] / s;
    f[9] = H[5] / s;
    f[10] = H[6] / qn;
    f[11] = H[7] / qn;
    f[12] = H[8] / qn;
    for (int k = 0; k < MLP_NIN && ok; ++k) ok = isfinite(f[k]) && isfinite((float)f[k]);
  }
  for (int k = 0; k < MLP_NIN; ++k) X[(size_t)c * MLP_NIN + k] = ok ? (float)f[k] : 0.0f;
  C.wnorm[c] = ok ? o[0] : 0.0;
  C.wnorm[(size_t)n + c] = ok ? o[4] : 0.0;
}

// S13 targets: HoT of cell r mod n normalised by input row r's rho and T_t
__global__ void k_cl_targets(Params P, CoupleParams C, const float* __restrict__ X, long long n_rows,
                             float* __restrict__ Y) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rows) return;
  const int n = P.n_cells;
  const int c = (int)(r % n);
  const double x0 = X[r * MLP_NIN], x4 = X[r * MLP_NIN + 4];
  bool ok = C.nbar[c] > 0.0 && x0 > 0.0 && x4 > 0.0;
  double y[MLP_NOUT];
  if (ok) {
    double o[6], H[12];
    hot_cell(P, C, c, o, H);
    const double s = x0 * x4, qn = s * sqrt(x4);
    y[0] = H[0] / s;
    y[1] = H[1] / s;
    y[2] = H[3] / s;
    y[3] = H[4] / s;
    y[4] = H[5] / s;
    y[5] = H[6] / qn;
    y[6] = H[7] / qn;
    y[7] = H[8] / qn;
    for (int k = 0; k < MLP_NOUT && ok; ++k) ok = isfinite(y[k]) && isfinite((float)y[k]);
  }
  for (int k = 0; k < MLP_NOUT; ++k) Y[r * MLP_NOUT + k] = ok ? (float)y[k] : 0.0f;
}

// S12 in the coupling: a cell with a valid window and a finite prediction
// within CLOSURE_YMAX takes the de-normalised prediction as its translational
// HoT; sigma_zz = -(sigma_xx + sigma_yy); q_r keeps the sampled value
__global__ void k_cl_apply(Params P, CoupleParams C, const float* __restrict__ Y) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = P.n_cells;
  if (c >= n) return;
  const double rho = C.wnorm[c], T = C.wnorm[(size_t)n + c];
  bool ok = rho > 0.0 && T > 0.0;
  double y[MLP_NOUT];
  for (int k = 0; k < MLP_NOUT; ++k) {
    y[k] = Y[(size_t)c * MLP_NOUT + k];
    ok = ok && isfinite(y[k]) && fabs(y[k]) <= CLOSURE_YMAX;
  }
  if (!ok) return;
  const double s = rho * T, qn = s * sqrt(T);
  double h[9];
  h[0] = __dmul_rn(y[0], s);
  h[1] = __dmul_rn(y[1], s);
  h[2] = -__dadd_rn(h[0], h[1]);
  h[3] = __dmul_rn(y[2], s);
  h[4] = __dmul_rn(y[3], s);
  h[5] = __dmul_rn(y[4], s);
  for (int q = 0; q < 3; ++q) h[6 + q] = __dmul_rn(y[5 + q], qn);
  for (int q = 0; q < 9; ++q) C.hot[(size_t)q * n + c] = h[q];
  atomicAdd(C.stats + 4, 1ull);
}

// one reconstruction layer (Sec. 3.2): a rejected cell with available face
// neighbours takes their mean, every neighbour with the same weight, and
// becomes available.  The mean is arithmetic, except that with recon = 1 the
// density and the temperatures take the logarithmic mean exp(mean ln) (the
// log-mean reconstruction of Sec. 6) where every contributing value is
// positive.  The first `passes` layers are the reconstruction (flag 2); later
// fill layers (fill >= 0: flag 3, counted in fillcnt[fill]) stop at the first
// layer after one that filled nothing
__global__ void k_cp_recon(Params P, CoupleParams C, const int* __restrict__ av_in, int* __restrict__ av_out,
                           int fill) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = P.n_cells;
  if (c >= n) return;
  if (fill > 0 && C.fillcnt[fill - 1] == 0) return;
  if (av_in[c]) {
    av_out[c] = 1;
    return;
  }
  double acc[18], lg[3] = {0.0, 0.0, 0.0};
  bool pos[3] = {true, true, true};
  for (int q = 0; q < 18; ++q) acc[q] = 0.0;
  int cnt = 0;
  for (int f = 0; f < 4; ++f) {
    const int nb = P.nbr[4 * (size_t)c + f];
    if (nb < 0 || !av_in[nb]) continue;
    for (int q = 0; q < 6; ++q) acc[q] += C.half[(size_t)q * n + nb];
    for (int q = 0; q < 12; ++q) acc[6 + q] += C.hot[(size_t)q * n + nb];
    if (C.recon == 1) {
      // density, translational and rotational temperature (rows 0, 4, 5)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double v = C.half[(size_t)(k == 0 ? 0 : 3 + k) * n + nb];
        if (v > 0.0)
          lg[k] += log(v);
        else
          pos[k] = false;
      }
    }
    cnt++;
  }
  av_out[c] = cnt > 0 ? 1 : 0;
  if (cnt == 0) return;
  for (int q = 0; q < 6; ++q) C.half[(size_t)q * n + c] = acc[q] / cnt;
  for (int q = 0; q < 12; ++q) C.hot[(size_t)q * n + c] = acc[6 + q] / cnt;
  if (C.recon == 1) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (pos[k]) C.half[(size_t)(k == 0 ? 0 : 3 + k) * n + c] = exp(lg[k] / cnt);
  }
  if (fill < 0) {
    C.flag[c] = 2.0;
    atomicAdd(C.stats + 1, 1ull);
  } else {
    C.flag[c] = 3.0;
    atomicAdd(C.fillcnt + fill, 1);
  }
}

// a cell that no accepted cell reaches within the reconstruction and fill
// layers (a region disconnected from every reliable cell) starts the solve
// from the configuration's initial state: density rho0, drift u_init,
// temperatures T0 (for an open domain the free stream), with zero HoT.  It
// keeps flag 0 and is not recalibrated.
__global__ void k_cp_unreached(Params P, CoupleParams C, const int* __restrict__ av) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = P.n_cells;
  if (c >= n || av[c]) return;
  C.half[c] = 1.0;
  for (int i = 0; i < 3; ++i) C.half[(size_t)(1 + i) * n + c] = C.u_ref[i];
  C.half[(size_t)4 * n + c] = 1.0;
  C.half[(size_t)5 * n + c] = 1.0;
  for (int q = 0; q < 12; ++q) C.hot[(size_t)q * n + c] = 0.0;
}

__device__ __forceinline__ void cons_from_prim(const CoupleParams& C, const double* Pp, double* U) {
  const double rho = Pp[0], uu = Pp[1] * Pp[1] + Pp[2] * Pp[2] + Pp[3] * Pp[3];
  const double er = C.dr > 0 ? 0.5 * C.dr * Pp[5] : 0.0;
  U[0] = rho;
  U[1] = rho * Pp[1];
  U[2] = rho * Pp[2];
  U[3] = rho * Pp[3];
  U[4] = rho * (1.5 * Pp[4] + 0.5 * uu + er);
  U[5] = rho * er;
}

__device__ __forceinline__ void prim_from_cons(const CoupleParams& C, const double* U, double* Pp) {
  const double rho = U[0];
  const double ir = 1.0 / rho;
  const double ux = U[1] * ir, uy = U[2] * ir, uz = U[3] * ir;
  const double er = C.dr > 0 ? U[5] * ir : 0.0;
  const double E = U[4] * ir;
  Pp[0] = rho;
  Pp[1] = ux;
  Pp[2] = uy;
  Pp[3] = uz;
  Pp[4] = (2.0 / 3.0) * (E - 0.5 * (ux * ux + uy * uy + uz * uz) - er);
  Pp[5] = C.dr > 0 ? (2.0 / C.dr) * er : Pp[4];
}

__global__ void k_cp_init_cons(Params P, CoupleParams C) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = P.n_cells;
  if (c >= n) return;
  double Pp[6], U[6];
  for (int q = 0; q < 6; ++q) Pp[q] = C.half[(size_t)q * n + c];
  cons_from_prim(C, Pp, U);
  for (int q = 0; q < 6; ++q) C.U[(size_t)q * n + c] = U[q];
}

// the primitives of the current state U, and its viscosity, sound speed and
// Mach number; the iteration limit N_m ends the solve here.  If the last
// Anderson combination was not positive in some cell, the state is the base
// step g(U) instead (U <- Gp; the following k_cp_reduce clears the history).
__global__ void k_cp_prim(Params P, CoupleParams C) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = P.n_cells;
  if (C.scal->done) return;
  if (C.scal->itc >= C.N_m) {
    if (c == 0) {
      C.scal->done = 1;
      C.scal->iters = C.N_m;
    }
    return;
  }
  if (c >= n) return;
  double U[6], Pp[6];
  const bool fb = C.scal->aabad != 0;
  for (int q = 0; q < 6; ++q) {
    const size_t k = (size_t)q * n + c;
    if (fb && (q < 5 || C.dr > 0)) C.U[k] = C.Gp[k];
    U[q] = C.U[k];
  }
  prim_from_cons(C, U, Pp);
  for (int q = 0; q < 6; ++q) C.prim[(size_t)q * n + c] = Pp[q];
  C.mu[c] = mu_nd(C, Pp[4]);
  const double cs = sqrt(C.gam * Pp[4]);
  C.snd[c] = cs;
  C.mach[c] = sqrt(Pp[1] * Pp[1] + Pp[2] * Pp[2] + Pp[3] * Pp[3]) / cs;
}

// total stress and heat fluxes per cell: NSF of the current state (its
// least-squares gradients and viscosity) + HoT
// (DI: diatomic; a monatomic gas has no rotational heat flux, whose terms are
// then left out: they are zero)
template <bool DI>
__global__ void k_cp_grad_stress(Params P, CoupleParams C) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = P.n_cells;
  if (c >= n || C.scal->done) return;
  double G[15];
  grad_cell<DI ? 5 : 4>(P, C, C.prim, c, G);
  double sig[6], qt[3], qr[3];
  nsf_mu(C, C.mu[c], G, sig, qt, qr);
  for (int q = 0; q < 6; ++q) C.S[(size_t)q * n + c] = sig[q] + C.hot[(size_t)q * n + c];
  for (int q = 0; q < 3; ++q) {
    C.S[(size_t)(6 + q) * n + c] = qt[q] + C.hot[(size_t)(6 + q) * n + c];
    if (DI) C.S[(size_t)(9 + q) * n + c] = qr[q] + C.hot[(size_t)(9 + q) * n + c];
  }
}

__device__ __forceinline__ void inv_flux(const double* Pp, const double* U, const double* N, double* F) {
  const double un = Pp[1] * N[0] + Pp[2] * N[1] + Pp[3] * N[2];
  const double p = Pp[0] * Pp[4];
  F[0] = U[0] * un;
  F[1] = U[1] * un + p * N[0];
  F[2] = U[2] * un + p * N[1];
  F[3] = U[3] * un + p * N[2];
  F[4] = (U[4] + p) * un;
  F[5] = U[5] * un;
}

constexpr int CPT = 128;

// Interior face flux (Rusanov inviscid flux plus the face-averaged stress and
// heat flux) seen from cell c with outward unit normal N, and the largest
// wave speed; from the other cell (normal -N) the flux is exactly -F.
template <bool DI>
__device__ __forceinline__ void interior_flux(const CoupleParams& C, const double* Pc, const double* Uc,
                                              const double* Pn, const double* Un, const double* Sc,
                                              const double* Sn, const double* N, double cl, double cr, double ml,
                                              double mr, double* F, double* lmo) {
  constexpr int NV = DI ? 6 : 5;  // conserved variables carried (rho e_r only for a diatomic gas)
  const double unl = Pc[1] * N[0] + Pc[2] * N[1] + Pc[3] * N[2];
  const double unr = Pn[1] * N[0] + Pn[2] * N[1] + Pn[3] * N[2];
  double FL[6], FR[6];
  {
    const double p = Pc[0] * Pc[4];
    FL[0] = Uc[0] * unl;
    FL[1] = Uc[1] * unl + p * N[0];
    FL[2] = Uc[2] * unl + p * N[1];
    FL[3] = Uc[3] * unl + p * N[2];
    FL[4] = (Uc[4] + p) * unl;
    FL[5] = DI ? Uc[5] * unl : 0.0;
  }
  {
    const double p = Pn[0] * Pn[4];
    FR[0] = Un[0] * unr;
    FR[1] = Un[1] * unr + p * N[0];
    FR[2] = Un[2] * unr + p * N[1];
    FR[3] = Un[3] * unr + p * N[2];
    FR[4] = (Un[4] + p) * unr;
    FR[5] = DI ? Un[5] * unr : 0.0;
  }
  const double lm = fmax(fabs(unl) + cl, fabs(unr) + cr);
  // low-Mach correction (Thornber et al. 2008): the dissipation acts on states
  // whose velocity jump is scaled by z = min(1, max(M_L, M_R)), so that at low
  // Mach the dissipation of shear and entropy waves scales with the flow speed
  const double z = fmin(1.0, fmax(ml, mr));
  // density jump: the acoustic part dp / c^2 kept, the entropy part scaled by
  // z (c^2 = gamma T of the face mean); the pressures unchanged, so the
  // conservative states follow from (rho', u', p) without T' = p / rho'
  const double pl = Pc[0] * Pc[4], pr = Pn[0] * Pn[4];
  const double c2 = C.gam * 0.5 * (Pc[4] + Pn[4]);
  const double dpc = (pl - pr) / c2;
  const double drho = dpc + z * ((Pc[0] - Pn[0]) - dpc);
  const double rm = 0.5 * (Pc[0] + Pn[0]);
  const double rl = rm + 0.5 * drho, rr = rm - 0.5 * drho;
  double UL[6], UR[6], ul2 = 0.0, ur2 = 0.0;
  UL[0] = rl;
  UR[0] = rr;
  for (int i = 1; i <= 3; ++i) {
    const double m = 0.5 * (Pc[i] + Pn[i]), h = 0.5 * z * (Pc[i] - Pn[i]);
    const double a = m + h, b = m - h;
    UL[i] = rl * a;
    UR[i] = rr * b;
    ul2 += a * a;
    ur2 += b * b;
  }
  const double erl = DI ? 0.5 * C.dr * Pc[5] : 0.0, err = DI ? 0.5 * C.dr * Pn[5] : 0.0;
  UL[4] = 1.5 * pl + rl * (0.5 * ul2 + erl);
  UR[4] = 1.5 * pr + rr * (0.5 * ur2 + err);
  UL[5] = rl * erl;
  UR[5] = rr * err;
  // the face's averages (half-sums) with their factors 1/2 taken out of the
  // sums: fewer FP64 multiplies
  for (int q = 0; q < NV; ++q) F[q] = 0.5 * ((FL[q] + FR[q]) - lm * (UR[q] - UL[q]));
  if (!DI) F[5] = 0.0;
  double ss[6], qts[3], qrs[3] = {0.0, 0.0, 0.0}, us[3];
  for (int q = 0; q < 6; ++q) ss[q] = Sc[q] + Sn[q];
  for (int q = 0; q < 3; ++q) {
    qts[q] = Sc[6 + q] + Sn[6 + q];
    if (DI) qrs[q] = Sc[9 + q] + Sn[9 + q];
    us[q] = Pc[1 + q] + Pn[1 + q];
  }
  const double sn0 = 0.5 * (ss[0] * N[0] + ss[3] * N[1] + ss[4] * N[2]);
  const double sn1 = 0.5 * (ss[3] * N[0] + ss[1] * N[1] + ss[5] * N[2]);
  const double sn2 = 0.5 * (ss[4] * N[0] + ss[5] * N[1] + ss[2] * N[2]);
  F[1] += sn0;
  F[2] += sn1;
  F[3] += sn2;
  if (DI) {
    F[4] += 0.5 * ((sn0 * us[0] + sn1 * us[1] + sn2 * us[2]) + (qts[0] + qrs[0]) * N[0] + (qts[1] + qrs[1]) * N[1] +
                   (qts[2] + qrs[2]) * N[2]);
    F[5] += 0.5 * (qrs[0] * N[0] + qrs[1] * N[1] + qrs[2] * N[2]);
  } else {
    F[4] += 0.5 * ((sn0 * us[0] + sn1 * us[1] + sn2 * us[2]) + qts[0] * N[0] + qts[1] * N[1] + qts[2] * N[2]);
  }
  *lmo = lm;
}

// flux of every interior face once, seen from its lower-index cell
template <bool DI>
__global__ void k_cp_face(Params P, CoupleParams C) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C.n_ifaces || C.scal->done) return;
  const int n = P.n_cells;
  const int c = C.fcell[i], f = C.fface[i];
  const int nb = P.nbr[4 * (size_t)c + f];
  const Plane64 pl = P.plane[4 * (size_t)c + f];
  const double N[3] = {pl.nx, pl.ny, pl.nz};
  constexpr int NV = DI ? 6 : 5, NS = DI ? 12 : 9;
  double Pc[6] = {}, Uc[6] = {}, Pn[6] = {}, Un[6] = {}, Sc[12] = {}, Sn[12] = {};
  for (int q = 0; q < NV; ++q) {
    Pc[q] = C.prim[(size_t)q * n + c];
    Uc[q] = C.U[(size_t)q * n + c];
    Pn[q] = C.prim[(size_t)q * n + nb];
    Un[q] = C.U[(size_t)q * n + nb];
  }
  for (int q = 0; q < NS; ++q) {
    Sc[q] = C.S[(size_t)q * n + c];
    Sn[q] = C.S[(size_t)q * n + nb];
  }
  const double cr = Pn[4] > 0 ? C.snd[nb] : sqrt(C.gam * 1e-12);
  double F[6], lm;
  interior_flux<DI>(C, Pc, Uc, Pn, Un, Sc, Sn, N, C.snd[c], cr, C.mach[c], C.mach[nb], F, &lm);
  for (int q = 0; q < NV; ++q) C.Ff[(size_t)q * C.n_ifaces + i] = F[q];
  C.lmf[i] = lm;
}

// residual and pseudo-time step of every cell from its face fluxes (the
// interior ones from k_cp_face, the boundary ones here): dtl = cfl V / sum_f
// A_f (lambda_f + 2 nu A_f / V), halved while the step would leave the cell
// a non-positive density or temperature; per-block partials of sum V |R|^2 (rho, rho
// u, rho E), of the mass after the base step sum V (rho + dtl R_rho) and of
// the current mass sum V rho
template <bool DI>
__global__ void __launch_bounds__(CPT) k_cp_flux(Params P, CoupleParams C) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = P.n_cells;
  if (C.scal->done) return;
  double rs = 0.0, mx = 0.0, m0 = 0.0;
  if (c < n) {
    double Pc[6], Uc[6];
    for (int q = 0; q < 6; ++q) {
      Pc[q] = C.prim[(size_t)q * n + c];
      Uc[q] = C.U[(size_t)q * n + c];
    }
    const double iL2 = C.iL2;
    const double V = C.vnd[c], iV = C.ivnd[c];
    double acc[6] = {0, 0, 0, 0, 0, 0};
    double lam_sum = 0.0;
    const double cc = C.snd[c];
    const double muc = C.mu[c];
    const double nu = 2.5 * muc / Pc[0];
    const double nu2 = 2.0 * nu * iV;  // viscous part of a face's wave speed, per unit area
    for (int f = 0; f < 4; ++f) {
      const double Ad = C.area[4 * (size_t)c + f];
      const double A = Ad * iL2;
      const int nb = P.nbr[4 * (size_t)c + f];
      double F[6];
      if (nb >= 0) {
        // the face's flux from k_cp_face, its sign for this cell folded into the area
        const int fi = C.cfid[4 * (size_t)c + f];
        const double sA = C.fcell[fi] == c ? A : -A;
        for (int q = 0; q < (DI ? 6 : 5); ++q) acc[q] += C.Ff[(size_t)q * C.n_ifaces + fi] * sA;
        lam_sum += A * (C.lmf[fi] + nu2 * A);
        continue;
      } else {
        const Plane64 pl = P.plane[4 * (size_t)c + f];
        const double N[3] = {pl.nx, pl.ny, pl.nz};
        const int kind = P.bc[P.bf[-1 - nb].bc].kind;
        if (kind >= 2) {
          // open boundary: Rusanov flux against the free stream (inflow) or
          // the cell's own state (outflow), no viscous terms
          double Pn[6], Un[6];
          const int b = P.bf[-1 - nb].bc;
          if (kind == 3) {
            for (int q = 0; q < 6; ++q) Pn[q] = Pc[q];
          } else {
            Pn[0] = C.bcn[b] * C.mass / C.rho0;
            Pn[1] = C.bcU[3 * b + 0] / C.c0;
            Pn[2] = C.bcU[3 * b + 1] / C.c0;
            Pn[3] = C.bcU[3 * b + 2] / C.c0;
            Pn[4] = C.bcT[b] / C.T0;
            Pn[5] = Pn[4];
          }
          cons_from_prim(C, Pn, Un);
          double FL[6], FR[6];
          inv_flux(Pc, Uc, N, FL);
          inv_flux(Pn, Un, N, FR);
          const double unl = Pc[1] * N[0] + Pc[2] * N[1] + Pc[3] * N[2];
          const double unr = Pn[1] * N[0] + Pn[2] * N[1] + Pn[3] * N[2];
          const double cl = cc, cr = sqrt(C.gam * (Pn[4] > 0 ? Pn[4] : 1e-12));
          const double lm = fmax(fabs(unl) + cl, fabs(unr) + cr);
          for (int q = 0; q < 6; ++q) F[q] = 0.5 * (FL[q] + FR[q]) - 0.5 * lm * (Un[q] - Uc[q]);
          lam_sum += A * (lm + nu2 * A);
        } else {
          // wall: no mass flux.  A diffuse wall closes the equations as an
          // isothermal no-slip wall: the cell's pressure and total stress (NSF
          // from gradients that take the wall velocity and temperature at the
          // face, plus the cell's HoT) plus the numerical friction below, the
          // work of both at the wall velocity and the cell's heat fluxes.  A
          // specular wall carries the cell's pressure only.
          const int b = P.bf[-1 - nb].bc;
          const double p = Pc[0] * Pc[4];
          F[0] = 0.0;
          if (kind == 0) {
            double Sc[12] = {};
            for (int q = 0; q < (DI ? 12 : 9); ++q) Sc[q] = C.S[(size_t)q * n + c];
            const double Uw[3] = {C.bcU[3 * b + 0] / C.c0, C.bcU[3 * b + 1] / C.c0, C.bcU[3 * b + 2] / C.c0};
            const double sn0 = Sc[0] * N[0] + Sc[3] * N[1] + Sc[4] * N[2];
            const double sn1 = Sc[3] * N[0] + Sc[1] * N[1] + Sc[5] * N[2];
            const double sn2 = Sc[4] * N[0] + Sc[5] * N[1] + Sc[2] * N[2];
            // the interior faces' dissipation against the mirrored ghost state
            // (velocity 2 U_w - u): a friction lambda z rho (U_w - u), lambda =
            // |u.n| + c, z = min(1, max(|u|/c, |U_w|/c)), its work done at U_w
            const double z = fmin(1.0, fmax(C.mach[c], sqrt(Uw[0] * Uw[0] + Uw[1] * Uw[1] + Uw[2] * Uw[2]) / cc));
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
          // wave speed of the wall face: |u.n| + c, as for the interior faces
          lam_sum += A * (fabs(Pc[1] * N[0] + Pc[2] * N[1] + Pc[3] * N[2]) + cc + nu2 * A);
        }
      }
      for (int q = 0; q < 6; ++q) acc[q] += F[q] * A;
    }
    double Rc[6];
    for (int q = 0; q < 6; ++q) Rc[q] = -acc[q] * iV;
    if (C.dr > 0) {
      const double T = (3.0 * Pc[4] + C.dr * Pc[5]) / (3.0 + C.dr);
      const double tau = muc / (Pc[0] * Pc[4]);
      Rc[5] += 0.5 * C.dr * Pc[0] * (T - Pc[5]) / (C.Zr * tau);
    } else {
      Rc[5] = 0.0;
    }
    for (int q = 0; q < 6; ++q) C.R[(size_t)q * n + c] = Rc[q];
    // the cell's base step, halved while it would leave a non-positive
    // density or temperature (at most 11 times, then no step)
    // (T_t > 0 tested without division: rho (rho E) - |rho u|^2 / 2 - rho (rho e_r) > 0)
    double dt = C.cfl * ldexp(1.0, -C.scal->halvings) * (V / lam_sum);
    for (int h = 0; h < 12; ++h) {
      double G[6];
      for (int q = 0; q < 6; ++q) G[q] = Uc[q] + dt * Rc[q];
      if (G[0] > 0.0 && G[0] * G[4] - 0.5 * (G[1] * G[1] + G[2] * G[2] + G[3] * G[3]) - G[0] * G[5] > 0.0) break;
      dt = h < 10 ? 0.5 * dt : 0.0;
    }
    C.dtl[c] = dt;
    for (int q = 0; q < 5; ++q) rs += V * Rc[q] * Rc[q];
    mx = V * (Uc[0] + dt * Rc[0]);
    m0 = V * Uc[0];
  }
  __shared__ double sr[3][CPT / 32];
  for (int o = 16; o > 0; o >>= 1) {
    rs += __shfl_xor_sync(0xffffffffu, rs, o);
    mx += __shfl_xor_sync(0xffffffffu, mx, o);
    m0 += __shfl_xor_sync(0xffffffffu, m0, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sr[0][threadIdx.x >> 5] = rs;
    sr[1][threadIdx.x >> 5] = mx;
    sr[2][threadIdx.x >> 5] = m0;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double a = sr[threadIdx.x][0];
    for (int w = 1; w < CPT / 32; ++w) a += sr[threadIdx.x][w];
    C.part[3 * blockIdx.x + threadIdx.x] = a;
  }
}

// residual norm, the stopping test and the mass-restoring factor of the base
// step (one block); the first iteration also records the initial mass
__global__ void k_cp_reduce(CoupleParams C, int nblocks) {
  if (C.scal->done) return;
  __shared__ double sh[3][1024];
  double a[3] = {0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
    for (int k = 0; k < 3; ++k) a[k] += C.part[3 * b + k];
  for (int k = 0; k < 3; ++k) sh[k][threadIdx.x] = a[k];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int k = 0; k < 3; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    CoupleScalars* S = C.scal;
    const int it = S->itc;
    const double res = sqrt(sh[0][0]);
    S->save = 0;
    S->revert = 0;
    if (it == 0) {
      S->res0 = res > 0 ? res : 1.0;
      S->M0 = sh[2][0];
      S->res_best = res;
      S->save = 1;
    }
    S->res = res;
    S->iters = it;
    if (res <= C.eps_m * S->res0) {
      S->done = 1;
    } else if (!(res <= 100.0 * S->res_best)) {
      // divergence (a non-finite residual or one 100 times the best): back to
      // the best iterate with half the CFL number (at most six times) and no
      // history; the next iteration starts there
      if (S->halvings >= 6) {
        S->done = 1;
      } else {
        S->revert = 1;
        S->halvings += 1;
        S->nh = 0;
        S->fresh = 1;
        S->aabad = 0;
        S->itc = it + 1;
      }
    } else {
      if (res < S->res_best) {
        S->res_best = res;
        S->save = 1;
      }
      S->mscale = C.closed ? S->M0 / sh[1][0] : 1.0;
      if (S->aabad) {  // the last combination fell back to the base step: restart the history
        S->nh = 0;
        S->aabad = 0;
      }
      S->itc = it + 1;
    }
  }
}

// Base step g(U) = s (U + dtl R) of every cell (s restores the total mass of
// a closed domain), f = g(U) - U; with Anderson acceleration the new
// differences dF_new, dG_new of f and g(U) go to ring slot `head`, and the
// block's partial (volume-weighted) dot products <dF_i, dF_new> of every held
// column i in age order (the new one last) and <dF_new, f> go to apart;
// without it U = g(U).  C.aab blocks loop over the cells, each thread
// accumulating its dot products in its own column of shared memory, so that
// the FP64 reduction across threads happens once per block and not once per
// cell.
template <bool DI>
__global__ void __launch_bounds__(CPT) k_aa_base(Params P, CoupleParams C) {
  constexpr int NV = DI ? 6 : 5;  // conserved variables carried (rho e_r only for a diatomic gas)
  __shared__ double red[AA_MAX + 1][CPT];
  __shared__ int sl[AA_MAX];
  const CoupleScalars* S = C.scal;
  if (S->done) return;
  const int n = P.n_cells;
  const int t = threadIdx.x;
  const int stride = gridDim.x * CPT;
  if (S->revert) {  // divergence: back to the best iterate, no step this iteration
    for (int c = blockIdx.x * CPT + t; c < n; c += stride)
      for (int q = 0; q < NV; ++q) C.U[(size_t)q * n + c] = C.Ub[(size_t)q * n + c];
    return;
  }
  const bool save = S->save;
  const int m = C.aa_m;
  const int it = S->itc - 1;
  const bool push = it > 0 && m > 0 && !S->fresh;
  const int head = S->head;
  const int nhn = push ? min(S->nh + 1, m) : 0;
  const int hn = (head + 1) % (m > 0 ? m : 1);
  const double s = S->mscale;
  if (push) {
    // slots of the held columns in age order; the new one (slot head) is last
    if (t < nhn - 1) sl[t] = ((hn - nhn + t) % m + m) % m;
    for (int i = 0; i <= nhn; ++i) red[i][t] = 0.0;
  }
  __syncthreads();
  for (int c = blockIdx.x * CPT + t; c < n; c += stride) {
    double f[6] = {0, 0, 0, 0, 0, 0}, dfn[6] = {0, 0, 0, 0, 0, 0};
    const double dt = C.dtl[c];
    for (int q = 0; q < NV; ++q) {
      const size_t k = (size_t)q * n + c;
      const double u = C.U[k];
      if (save) C.Ub[k] = u;
      double gx = u + dt * C.R[k];
      if (C.closed) gx *= s;
      if (m == 0) {
        C.U[k] = gx;
        continue;
      }
      const double fq = gx - u;
      if (push) {
        const size_t h = ((size_t)head * 6 + q) * n + c;
        dfn[q] = fq - C.fp[k];
        C.dF[h] = dfn[q];
        C.dG[h] = gx - C.Gp[k];
      }
      C.fp[k] = fq;
      C.Gp[k] = gx;
      f[q] = fq;
    }
    if (!push) continue;
    const double V = C.vnd[c];
    double dv[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) dv[q] = V * dfn[q];
    // the held columns are not written by this kernel (the new one goes to
    // slot head, which is not among them)
#pragma unroll 4
    for (int i = 0; i < nhn - 1; ++i) {
      const double* col = C.dF + (size_t)sl[i] * 6 * n + c;
      double a = red[i][t];
#pragma unroll
      for (int q = 0; q < NV; ++q) a = fma(__ldg(col + (size_t)q * n), dv[q], a);
      red[i][t] = a;
    }
    double a = red[nhn - 1][t], b = red[nhn][t];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      a = fma(dfn[q], dv[q], a);
      b = fma(dv[q], f[q], b);
    }
    red[nhn - 1][t] = a;
    red[nhn][t] = b;
  }
  if (!push) return;
  __syncthreads();
  const int lane = t & 31, warp = t >> 5;
  for (int i = warp; i <= nhn; i += CPT / 32) {
    double a = 0.0;
#pragma unroll
    for (int r = 0; r < CPT; r += 32) a += red[i][r + lane];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) C.apart[(size_t)(i < nhn ? i : AA_MAX) * gridDim.x + blockIdx.x] = a;
  }
}

// Anderson coefficients (one block): the block partials summed, the new
// column's row of the Gram matrix stored, then gamma minimising
// |f - dF gamma| from the normal equations of the columns scaled to unit
// norm with 1e-10 added to the diagonal, by a right-looking Cholesky over the
// block (thread (i, j) owning entry (i, j)) and substitutions in one warp
// (lane i owning row i); a failed factorisation uses no column
__global__ void k_aa_solve(CoupleParams C, int nblocks) {
  __shared__ double val[AA_MAX + 1];
  __shared__ double L[AA_MAX][AA_MAX + 1];
  __shared__ int sl[AA_MAX];
  CoupleScalars* S = C.scal;
  if (S->done || S->revert) return;
  const int m = C.aa_m;
  const int it = S->itc - 1;
  const bool push = it > 0 && !S->fresh;
  const int head = S->head;
  const int nhn = push ? min(S->nh + 1, m) : S->nh;
  const int hn = push ? (head + 1) % m : head;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int k = nhn;
  // the stored Gram matrix in age order (before the new row arrives; its
  // row and column are overwritten below), loaded by the whole block
  if (threadIdx.x < AA_MAX) sl[threadIdx.x] = threadIdx.x < k ? ((hn - k + (int)threadIdx.x) % m + m) % m : 0;
  __syncthreads();
  AAState* A = C.aa;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int i = e / k, j = e - i * k;
    L[i][j] = A->H[sl[i] * AA_MAX + sl[j]];
  }
  // block partials, four independent sums per lane: <dF_i, dF_new> at j < k,
  // <dF_new, f> at j = AA_MAX
  for (int j = warp; j <= AA_MAX; j += nw) {
    if (!push || (j < AA_MAX && j >= nhn)) continue;
    const double* pj = C.apart + (size_t)j * nblocks;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int b = lane;
    for (; b + 96 < nblocks; b += 128) {
      a0 += pj[b];
      a1 += pj[b + 32];
      a2 += pj[b + 64];
      a3 += pj[b + 96];
    }
    for (; b < nblocks; b += 32) a0 += pj[b];
    double a = (a0 + a1) + (a2 + a3);
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) val[j] = a;
  }
  __syncthreads();
  if (push && threadIdx.x < k) {  // the new column (newest, age k - 1) against every held column
    const int i = threadIdx.x;
    const double h = val[i];
    A->H[head * AA_MAX + sl[i]] = h;
    A->H[sl[i] * AA_MAX + head] = h;
    L[k - 1][i] = h;
    L[i][k - 1] = h;
    // b_i = <dF_i, f_k> = <dF_i, f_{k-1}> + <dF_i, dF_new>; the new column's is computed
    A->b[sl[i]] = i == k - 1 ? val[AA_MAX] : A->b[sl[i]] + h;
  }
  if (threadIdx.x == 0) {
    S->head = hn;
    S->nh = k;
    S->fresh = 0;
  }
  __syncthreads();
  // scaled, regularised normal matrix: thread (ti, tq) owns entry (ti, tq)
  __shared__ double scs[AA_MAX], inv[AA_MAX];
  __shared__ int okf;
  const int ti = threadIdx.x >> 5, tq = threadIdx.x & 31;
  if (threadIdx.x < k) {
    const double d = L[threadIdx.x][threadIdx.x];
    scs[threadIdx.x] = d > 0 ? rsqrt(d) : 0.0;
  }
  __syncthreads();
  if (ti < k && tq < k) L[ti][tq] = L[ti][tq] * scs[ti] * scs[tq] + (ti == tq ? 1e-10 : 0.0);
  __syncthreads();
  // right-looking Cholesky: every entry receives its updates in the order of
  // the left-looking form (column 0 first), then the division by its pivot
  // (pivots by rsqrt, so that the column is scaled by a product: FP64
  // division and square root are long dependent sequences on this part)
  bool ok = true;
  for (int j = 0; j < k; ++j) {
    if (threadIdx.x == 0) {
      const double d = L[j][j];
      okf = d > 0;
      if (d > 0) {
        const double r = rsqrt(d);
        inv[j] = r;
        L[j][j] = d * r;
      }
    }
    __syncthreads();
    if (!okf) {
      ok = false;
      break;
    }
    if (tq == j && ti > j && ti < k) L[ti][j] *= inv[j];
    __syncthreads();
    if (ti > j && ti < k && tq > j && tq <= ti) L[ti][tq] -= L[ti][j] * L[tq][j];
    __syncthreads();
  }
  if (warp != 0) return;
  const double sci = lane < k ? scs[lane] : 0.0;
  const double bi = lane < k ? A->b[sl[lane]] * sci : 0.0;
  if (ok) {
    // L y = b, then L^T g = y, column-oriented: lane i holds entry i of the
    // right-hand side; once y_j (g_j) is known every later lane subtracts its
    // multiple, so each step is one broadcast and one multiply-add
    double r = bi;
    for (int j = 0; j < k; ++j) {
      const double y = __shfl_sync(0xffffffffu, r, j) * inv[j];
      if (lane == j) r = y;
      else if (lane > j && lane < k) r = fma(-L[lane][j], y, r);
    }
    for (int j = k - 1; j >= 0; --j) {
      const double g = __shfl_sync(0xffffffffu, r, j) * inv[j];
      if (lane == j) r = g;
      else if (lane < j) r = fma(-L[j][lane], g, r);
    }
    if (lane < k) {
      A->gam[lane] = r * sci;
      A->slot[lane] = sl[lane];
    }
  }
  if (lane == 0) S->k = ok ? k : 0;
}

// the combination U = g(U_k) - sum_i gamma_i dG_i; a cell whose combined
// density or temperature is not positive flags the fallback
template <bool DI>
__global__ void __launch_bounds__(CPT) k_aa_update(Params P, CoupleParams C) {
  constexpr int NV = DI ? 6 : 5;
  __shared__ double gam[AA_MAX];
  __shared__ int sl[AA_MAX];
  if (C.scal->done || C.scal->revert) return;
  const int k = C.scal->k;
  if (threadIdx.x < k) {
    gam[threadIdx.x] = C.aa->gam[threadIdx.x];
    sl[threadIdx.x] = C.aa->slot[threadIdx.x];
  }
  __syncthreads();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = P.n_cells;
  if (c >= n) return;
  double U[6] = {0, 0, 0, 0, 0, 0}, Pp[6];
#pragma unroll
  for (int q = 0; q < NV; ++q) U[q] = C.Gp[(size_t)q * n + c];
  // column by column, every component's sum in the order j = 0, 1, ...
#pragma unroll 2
  for (int j = 0; j < k; ++j) {
    const double* col = C.dG + (size_t)sl[j] * 6 * n + c;
    const double g = gam[j];
#pragma unroll
    for (int q = 0; q < NV; ++q) U[q] -= g * __ldg(col + (size_t)q * n);
  }
#pragma unroll
  for (int q = 0; q < NV; ++q) C.U[(size_t)q * n + c] = U[q];
  prim_from_cons(C, U, Pp);
  if (!(Pp[0] > 0.0 && Pp[4] > 0.0)) C.scal->aabad = 1;
}

__global__ void k_cp_final(Params P, CoupleParams C) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = P.n_cells;
  if (c == 0 && !C.scal->done) C.scal->iters = C.scal->itc;
  if (c >= n) return;
  double U[6], Pp[6];
  // the best iterate if the last one is worse (a stop at N_m after a rise
  // of the residual, or a divergence); else a pending fallback (N_m reached
  // right after a failed combination) or the last iterate
  const bool best = !(C.scal->res <= C.scal->res_best);
  const bool fb = C.scal->aabad != 0;
  for (int q = 0; q < 6; ++q) {
    const size_t k = (size_t)q * n + c;
    const bool carried = q < 5 || C.dr > 0;
    U[q] = best && carried ? C.Ub[k] : fb && carried ? C.Gp[k] : C.U[k];
  }
  prim_from_cons(C, U, Pp);
  for (int q = 0; q < 6; ++q) C.newst[(size_t)q * n + c] = Pp[q];
  if (!(Pp[0] > 0.0) || !(Pp[4] > 0.0) || !isfinite(Pp[0]) || !isfinite(Pp[4])) C.scal->bad = 1;
}

// ---------------------------------------------------------------------------
// S11 recalibration of the particles of accepted cells
// ---------------------------------------------------------------------------

struct RecalCell {
  float ua[3], ub[3], sc, fr;
  double rn;
  bool on;
};

// b = the cell's own (moving-average) state, a = the solved state; the number
// ratio is taken against the density of the N_c particles the cell holds now
// (rho_N = m F_N N_c / V), so the expected count afterwards is rho_a V / (m F_N)
__device__ __forceinline__ RecalCell recal_cell(const Params& P, const CoupleParams& C, int c, int n, int Nc) {
  RecalCell r;
  r.on = C.flag[c] == 1.0;
  const double b4 = C.own[(size_t)4 * n + c], a4 = C.newst[(size_t)4 * n + c];
  double rt = a4 / b4;
  rt = rt < 0.25 ? 0.25 : rt > 4.0 ? 4.0 : rt;
  double rr = C.dr > 0 ? C.newst[(size_t)5 * n + c] / C.own[(size_t)5 * n + c] : 1.0;
  rr = rr < 0.25 ? 0.25 : rr > 4.0 ? 4.0 : rr;
  const double rho_N = C.mass * C.FN * (double)Nc / P.vol[c] / C.rho0;
  double rn = Nc > 0 ? C.newst[c] / rho_N : 1.0;
  r.rn = rn < 0.5 ? 0.5 : rn > 2.0 ? 2.0 : rn;
  r.sc = (float)sqrt(rt);
  r.fr = (float)rr;
  for (int i = 0; i < 3; ++i) {
    r.ua[i] = (float)(C.newst[(size_t)(1 + i) * n + c] * C.c0);
    r.ub[i] = (float)(C.own[(size_t)(1 + i) * n + c] * C.c0);
  }
  return r;
}

// one warp per cell: rescale velocities and rotational energies in place,
// decide deletion (mc = -1) or cloning (flag in cl[slot])
__global__ void k_recal_decide(Params P, CoupleParams C, Buf CUR, int* __restrict__ cl, uint32_t sub) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  const int n = P.n_cells;
  for (int c = gw; c < n; c += nw) {
    const int lo = P.cs[c], hi = P.cs[c + 1];
    const RecalCell r = recal_cell(P, C, c, n, hi - lo);
    int stay = 0;
    for (int p = lo + lane; p < hi; p += 32) {
      int clone = 0;
      bool keep = true;
      if (r.on) {
        // v' = u_a + (v - u_b) sc, evaluated as written (no fused multiply-add)
        float* vp = CUR.vel + 3 * (size_t)p;
        for (int i = 0; i < 3; ++i) vp[i] = __fadd_rn(r.ua[i], __fmul_rn(__fsub_rn(vp[i], r.ub[i]), r.sc));
        if (C.dr > 0) CUR.Ir[p] = __fmul_rn(CUR.Ir[p], r.fr);
        uint32_t w[4];
        philox((uint32_t)p, sub, 0u, 0u, P.seed_lo, P.seed_hi ^ (RP_RECAL << 24), w);
        const double R = u01d(w[0], w[1]);
        if (r.rn < 1.0) {
          if (R < 1.0 - r.rn) keep = false;
        } else if (r.rn > 1.0 && R < r.rn - 1.0) {
          clone = 1;
        }
      }
      CUR.mc[p] = keep ? c : -1;
      cl[p] = clone;
      stay += keep ? 1 : 0;
      if (!keep) atomicAdd(C.stats + 3, 1ull);
    }
    for (int o = 16; o > 0; o >>= 1) stay += __shfl_xor_sync(0xffffffffu, stay, o);
    if (lane == 0) {
      P.nst[c] = stay;
      P.sbase[c] = lo;
      P.nold[c] = hi - lo;
    }
  }
}

// exclusive scan of the clone flags over the particles (two kernels)
constexpr int RS = 1024 * 4;
__global__ void __launch_bounds__(1024) k_recal_reduce(const int* __restrict__ cl, int N, int* part) {
  int t = 0;
  for (int i = blockIdx.x * RS + threadIdx.x; i < min(N, (int)(blockIdx.x + 1) * RS); i += 1024) t += cl[i];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  __shared__ int sh[32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    int a = 0;
    for (int w = 0; w < 32; ++w) a += sh[w];
    part[blockIdx.x] = a;
  }
}

__global__ void __launch_bounds__(1024) k_recal_scan(int* __restrict__ cl, int N, const int* part, int nb,
                                                     int* total) {
  __shared__ int sh[32];
  __shared__ int s_off;
  int p = 0;
  for (int b = threadIdx.x; b < (int)blockIdx.x; b += 1024) p += part[b];
  for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = p;
  __syncthreads();
  if (threadIdx.x == 0) {
    int a = 0;
    for (int w = 0; w < 32; ++w) a += sh[w];
    s_off = a;
  }
  __syncthreads();
  const int i0 = blockIdx.x * RS + threadIdx.x * 4;
  int v[4], loc = 0;
  for (int u = 0; u < 4; ++u) {
    v[u] = i0 + u < N ? cl[i0 + u] : 0;
    loc += v[u];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int inc = loc;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  __syncthreads();
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
  int e = s_off + inc - loc + (warp > 0 ? sh[warp - 1] : 0);
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + u;
    if (i < N) cl[i] = v[u] ? e : -1;
    e += v[u];
    if (i == N - 1) *total = e;
  }
}

// clones at slots N + (their rank), uniform point in the parent's cell
__global__ void k_recal_clone(Params P, CoupleParams C, Buf CUR, const int* __restrict__ cl, int N, uint32_t sub) {
  const int n = P.n_cells;
  const int total = *C.clone_total;
  long long hi = (long long)N + total;
  if (hi > P.cap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(P.status, ST_CAPACITY);
    hi = P.cap;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    P.state[1] = N;
    P.state[2] = (int)hi;
  }
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    for (int p = P.cs[c]; p < P.cs[c + 1]; ++p) {
      const int r = cl[p];
      if (r < 0) continue;
      const long long q = (long long)N + r;
      if (q >= hi) continue;
      uint32_t w[4], w2[4];
      philox((uint32_t)p, sub, 0u, 1u, P.seed_lo, P.seed_hi ^ (RP_RECAL << 24), w);
      philox((uint32_t)p, sub, 0u, 2u, P.seed_lo, P.seed_hi ^ (RP_RECAL << 24), w2);
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
      const int* tv = P.tets + 4 * (size_t)c;
      const double* A = P.nodes + 3 * (size_t)tv[0];
      const double* B = P.nodes + 3 * (size_t)tv[1];
      const double* Cc = P.nodes + 3 * (size_t)tv[2];
      const double* D = P.nodes + 3 * (size_t)tv[3];
      // uniform point in the tet, evaluated as written (no fused multiply-add)
      double xs[3];
      for (int i = 0; i < 3; ++i)
        xs[i] = __dadd_rn(__dadd_rn(__dadd_rn(A[i], __dmul_rn(s, __dsub_rn(B[i], A[i]))),
                                    __dmul_rn(tt, __dsub_rn(Cc[i], A[i]))),
                          __dmul_rn(u, __dsub_rn(D[i], A[i])));
      CUR.pos[3 * (size_t)q] = xs[0];
      CUR.pos[3 * (size_t)q + 1] = xs[1];
      CUR.pos[3 * (size_t)q + 2] = xs[2];
      for (int i = 0; i < 3; ++i) CUR.vel[3 * (size_t)q + i] = CUR.vel[3 * (size_t)p + i];
      if (C.dr > 0) CUR.Ir[q] = CUR.Ir[p];
      CUR.mc[q] = c;
      atomicAdd(P.na + c, 1);
      atomicAdd(C.stats + 2, 1ull);
    }
  }
}

int nb_for(int n, int t) { return (n + t - 1) / t; }
}  // namespace

void launch_couple_s9(const Params& P, const CoupleParams& C, int passes, const float* ypred, int** av,
                      cudaStream_t s) {
  const int n = P.n_cells, nb = nb_for(n, CPT);
  k_cp_extract<<<nb, CPT, 0, s>>>(P, C, P.phi_ewma, 1.0);
  k_cp_grad<<<nb, CPT, 0, s>>>(P, C, C.own, C.grad);
  k_cp_hot<<<nb, CPT, 0, s>>>(P, C);
  if (ypred) {
    k_cl_apply<<<nb, CPT, 0, s>>>(P, C, ypred);
    ++g_launches;
  }
  int* a = C.avail;
  int* b = C.avail2;
  for (int q = 0; q < passes; ++q) {
    k_cp_recon<<<nb, CPT, 0, s>>>(P, C, a, b, -1);
    int* t = a;
    a = b;
    b = t;
  }
  g_launches += 3 + passes;
  *av = a;
  // fill layers: rejected cells beyond the reconstruction layers still need a
  // state for the solve; they are filled the same way, layer by layer
  launch_couple_fill(P, C, 0, DIG_FILL_CHUNK, av, s);
}

// A layer that returns early (the previous one filled nothing) leaves its
// output array as it was; both arrays then already hold the same
// availability, since a layer that fills nothing copies it unchanged, so the
// alternation below stays exact.
void launch_couple_fill(const Params& P, const CoupleParams& C, int q0, int q1, int** av, cudaStream_t s) {
  const int n = P.n_cells, nb = nb_for(n, CPT);
  int* a = *av;
  int* b = a == C.avail ? C.avail2 : C.avail;
  for (int q = q0; q < q1; ++q) {
    k_cp_recon<<<nb, CPT, 0, s>>>(P, C, a, b, q);
    int* t = a;
    a = b;
    b = t;
  }
  g_launches += q1 - q0;
  *av = a;
}

void launch_couple_unreached(const Params& P, const CoupleParams& C, const int* av, cudaStream_t s) {
  const int n = P.n_cells, nb = nb_for(n, CPT);
  k_cp_unreached<<<nb, CPT, 0, s>>>(P, C, av);
  g_launches += 1;
}

void launch_couple_s10_init(const Params& P, const CoupleParams& C, cudaStream_t s) {
  const int n = P.n_cells, nb = nb_for(n, CPT);
  k_cp_init_cons<<<nb, CPT, 0, s>>>(P, C);
  g_launches += 1;
}

template <bool DI>
static long long s10_iteration(const Params& P, const CoupleParams& C, int nb, cudaStream_t s) {
  k_cp_prim<<<nb, CPT, 0, s>>>(P, C);
  k_cp_grad_stress<DI><<<nb, CPT, 0, s>>>(P, C);
  if (C.n_ifaces > 0) k_cp_face<DI><<<nb_for(C.n_ifaces, CPT), CPT, 0, s>>>(P, C);
  k_cp_flux<DI><<<nb, CPT, 0, s>>>(P, C);
  k_cp_reduce<<<1, 1024, 0, s>>>(C, nb);
  k_aa_base<DI><<<C.aab, CPT, 0, s>>>(P, C);
  long long k = C.n_ifaces > 0 ? 6 : 5;
  if (C.aa_m > 0) {
    k_aa_solve<<<1, 1024, 0, s>>>(C, C.aab);
    k_aa_update<DI><<<nb, CPT, 0, s>>>(P, C);
    k += 2;
  }
  return k;
}

long long launch_couple_s10_iters(const Params& P, const CoupleParams& C, int iters, cudaStream_t s) {
  const int nb = nb_for(P.n_cells, CPT);
  long long k = 0;
  for (int it = 0; it < iters; ++it) k += C.dr > 0 ? s10_iteration<true>(P, C, nb, s) : s10_iteration<false>(P, C, nb, s);
  return k;
}

void launch_couple_s10_final(const Params& P, const CoupleParams& C, cudaStream_t s) {
  k_cp_final<<<nb_for(P.n_cells, CPT), CPT, 0, s>>>(P, C);
  g_launches += 1;
}

void launch_couple_s11(const Params& P, const CoupleParams& C, const Buf& cur, int N, uint32_t sub, int* cl,
                       cudaStream_t s) {
  const int n = P.n_cells;
  k_recal_decide<<<nb_for(n * 32, 256), 256, 0, s>>>(P, C, cur, cl, sub);
  const int nbr = (N + RS - 1) / RS;
  if (N > 0) {
    k_recal_reduce<<<nbr, 1024, 0, s>>>(cl, N, C.rpart);
    k_recal_scan<<<nbr, 1024, 0, s>>>(cl, N, C.rpart, nbr, C.clone_total);
  }
  k_recal_clone<<<nb_for(n, 256), 256, 0, s>>>(P, C, cur, cl, N, sub);
  g_launches += N > 0 ? 4 : 2;
}

void launch_closure_features(const Params& P, const CoupleParams& C, const double* phi, double cnt, float* X,
                             cudaStream_t s) {
  const int n = P.n_cells, nb = nb_for(n, CPT);
  k_cp_extract<<<nb, CPT, 0, s>>>(P, C, phi, cnt);
  k_cp_grad<<<nb, CPT, 0, s>>>(P, C, C.own, C.grad);
  k_cl_features<<<nb, CPT, 0, s>>>(P, C, X);
  g_launches += 3;
}

void launch_closure_targets(const Params& P, const CoupleParams& C, const double* phi, double cnt, const float* X,
                            long long n_rows, float* Y, cudaStream_t s) {
  const int n = P.n_cells, nb = nb_for(n, CPT);
  k_cp_extract<<<nb, CPT, 0, s>>>(P, C, phi, cnt);
  k_cp_grad<<<nb, CPT, 0, s>>>(P, C, C.own, C.grad);
  g_launches += 2;
  if (n_rows > 0) {
    k_cl_targets<<<(unsigned)((n_rows + 255) / 256), 256, 0, s>>>(P, C, X, n_rows, Y);
    ++g_launches;
  }
}

size_t couple_part_count(int n_cells) { return 3 * (size_t)nb_for(n_cells, CPT) + 2; }
size_t couple_apart_count(int n_cells) { return (size_t)(AA_MAX + 1) * nb_for(n_cells, CPT); }

int couple_aa_blocks(int n_cells) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max(1, std::min(nb_for(n_cells, CPT), 4 * sms));
}

}  // namespace dig
