// dig_internal.h -- structures shared by the host API (dig_api.cu) and the
// kernels (dig_kernels.cu).  Not part of the public ABI.
#pragma once
#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

namespace dig {

constexpr int NPHI = 17;  // summation variables per cell (13 monatomic + 4 rotational)
constexpr int NMAC = 20;  // derived moments per cell
constexpr int N_COUNTERS = 9;

// pass flags of the cell kernel
enum : int { PASS_COLLIDE = 1, PASS_MOVE = 2 };
// sampling flags (same bits as the public DIG_* flags)
enum : int { S_EWMA = 1, S_WINDOW = 2, S_CUMUL = 4, S_PAIRS = 8, S_INST = 16, S_WALLFLUX = 32 };
// device status bits
enum : int { ST_CAPACITY = 2, ST_PAIRS_FULL = 4 };
// counters
enum : int { C_STEPS, C_CAND, C_COLL, C_CROSS, C_WALL, C_REMOVED, C_INJECTED, C_STUCK, C_LB };
// random-stream purposes: key = (seed_lo, seed_hi ^ purpose << 24)
enum : uint32_t { RP_INIT_POS = 1, RP_INIT_VEL = 2, RP_WALL = 3, RP_INJECT = 4, RP_COLL = 5,
                  RP_DIR = 6, RP_LB = 7, RP_RECAL = 8, RP_MLP_INIT = 9 };
// learned closure
constexpr int MLP_NIN = 13, MLP_NOUT = 8, MLP_NPARAM = 9736;
constexpr double CLOSURE_YMAX = 4.0;

// FP64 face plane: outward unit normal (nx, ny, nz) and offset d, n.x = d on the face
struct __align__(32) Plane64 {
  double nx, ny, nz, d;
};

struct BCDev {
  int kind;
  float sigma;  // sqrt(k T / m)
  float T;
  float U[3];
};

struct BFaceDev {
  int bc;
  float nrm[3], t1[3], t2[3];
};

// a free-stream inflow face: its boundary face, tet and local face, corners,
// expected injections per step and the constants of the inflow law
struct InflowDev {
  int bface, tet, face, pad;
  double a[3], b[3], c[3];
  double expn;
  float s, p1, invb, sig, ut1, ut2;
};

// one particle buffer, structure of arrays; x,y,z and vx,vy,vz are contiguous
// blocks of `cap` elements each
struct Buf {
  double* pos;  // [cap][3] positions x, y, z of each slot, one 24-byte record per particle
  float* vel;   // [cap][3] velocities vx, vy, vz, one 12-byte record per particle
  float* Ir;
  int* mc;  // cell of the particle at each slot after the move that wrote it (-1: removed)
};

struct Params {
  // mesh
  int n_cells, n_bf, max_cross, rot_dof;
  const int* nbr;           // [4n]: >= 0 neighbour, < 0: -1 - boundary face
  const signed char* nbrf;  // [4n] matching face in the neighbour
  const Plane64* plane;     // [4n]
  const float4* plane32;    // FP32 copy used by the inside filter
  const double* fdtv;       // [n] F_N dt / V
  const double* vol;        // [n]
  const double* cumvol;     // [n] running sum of volumes
  const double* nodes;      // [n_nodes][3] (initial sampling only)
  const int* tets;          // [n][4]
  const BFaceDev* bf;
  const BCDev* bc;
  double* bflux;            // [5 n_bf]
  int n_in;                 // inflow faces
  const InflowDev* inflow;  // [n_in]
  double* inj_rem;          // [n_in] carried fractional injection counts
  int* inj_cnt;             // [n_in] injections of the current step
  int* inj_off;             // [n_in + 1] their exclusive scan
  float margin;             // FP32 filter margin (see track())
  double dt;
  double mass_fn;           // m F_N (wall flux bookkeeping)
  double fn_kb;             // F_N k_B
  // gas constants in FP32
  uint32_t seed_lo, seed_hi;
  float c_vhs, one_m_omega, p_inel, lb_exp, hmr;
  float inv_alpha;          // 1 / alpha of the VSS scattering law (alpha != 1)
  int local_acc;            // 1: rejected cells accumulate (acc_w)
  double* acc_w;            // [n] samples a cell's average stands for in the local accumulation state (0: moving average)
  int vss;                  // 1: VSS scattering, 0: VHS (isotropic)
  float T_init, sigma_init, u0[3];
  // per-cell grouping and sort state
  int* cs;      // [n+1] start of each cell in the current grouping
  int* as;      // [n+1] start of each cell's arrivals in aq
  int* nst;     // [n] stayers count
  int* sbase;   // [n] first slot of the cell's range in the last written buffer
  int* nold;    // [n] particles of the cell in the last written buffer
  int* na;      // [n] arrivals counted for the next grouping
  int* fill;    // [n] scatter cursor
  int* aq;      // [cap] arrival lists: buffer slot of each arrival
  float* cmax;  // [n] (sigma c_r)_max
  double* rem;  // [n] NTC remainder
  double* phi_inst;  // [NPHI][n]
  double* phi_ewma;
  double* phi_win;
  double* phi_cum;
  unsigned long long* counters;  // [16]
  int* status;
  int* state;   // [0] N, [1] extra_lo, [2] extra_hi, [3] track-queue length
  int* tq;      // [2 cap] track queue: (output slot, input slot) of each particle left to k_track
  int* src;     // [cap] slot map of the pass: input slot of the particle at each output slot
  int* scan_part;
  int* pairs;   // [4 * pair_cap]
  unsigned char* pacc;
  unsigned long long* pair_count;
  long long pair_cap;
  long long cap;
};

// DIG coupling state (dig_couple.cu); arrays are [component][cell].
// The scalars of one solve; cleared before every coupling.
struct CoupleScalars {
  double res0, res;
  double res_best;  // the smallest residual so far (its state in CoupleParams::Ub)
  double M0;      // total mass of the initial state (closed domains)
  double mscale;  // mass-restoring factor of the current base step (1 for open domains)
  int iters, done, bad;
  int itc;        // index of the next iteration
  int head, nh;   // Anderson history: next slot to write, columns held
  int aabad;      // a combined state was not positive: fall back to the base step
  int k;          // columns used by the current combination (0: base step)
  int halvings;   // of the CFL number after divergences (the step scale is 2^-halvings)
  int save;       // this iteration's state is the best so far: copy it to Ub
  int revert;     // divergence: this iteration returns to Ub instead of stepping
  int fresh;      // no previous f to difference with (after a return to Ub)
};

// most Anderson-acceleration columns
constexpr int AA_MAX = 32;

// Anderson-acceleration state of the synthetic solve: Gram matrix of the
// stored residual differences (indexed by ring slot), and the coefficients
// and slots of the current combination in age order (oldest first)
struct AAState {
  double H[AA_MAX * AA_MAX];
  double b[AA_MAX];  // <dF_i, f_k> by ring slot
  double gam[AA_MAX];
  int slot[AA_MAX];
};

// most fill layers after the reconstruction layers (see k_cp_recon), issued
// in chunks of DIG_FILL_CHUNK; the host stops after a chunk whose last layer
// filled nothing
constexpr int DIG_FILL_LAYERS = 1024;
constexpr int DIG_FILL_CHUNK = 64;

struct CoupleParams {
  double L0, T0, rho0, c0, Kn, omega, gam, dr, Zr, mass, FN, kB, KnD_max, wall_t;
  double acc_w0;       // min(m, n_a): the samples a moving average stands for at this coupling
  double u_ref[3];     // initial drift / c0: velocity of the state of unreached cells
  double iL2;          // 1 / L0^2
  const double* vnd;   // [n] cell volumes / L0^3
  const double* ivnd;  // [n] L0^3 / cell volumes
  const double* area;  // [4n] face areas
  const double* lsqw;  // [12][n] least-squares gradient weights (M^-1 d_f)_i at row 3f + i, nondimensional
  const double* bcU;   // [3 n_bcs]
  const double* bcT;   // [n_bcs]
  const double* bcn;   // [n_bcs]
  double *own, *sd, *grad, *half, *hot, *newst, *flag, *nbar, *U, *prim, *S, *R, *part, *mu, *snd;
  double* mach;  // [n] |u| / c of the current state
  int *avail, *avail2;
  int n_ifaces;          // interior faces (each once)
  int recon;             // reconstruction mean of density and temperatures: 0 arithmetic, 1 logarithmic
  const int* fcell;      // [n_ifaces] lower-index cell of each interior face
  const int* fface;      // [n_ifaces] its local face
  const int* cfid;       // [4n] interior face of (cell, local face), -1 on the boundary
  double *Ff, *lmf;      // [6][n_ifaces] face fluxes, [n_ifaces] wave speeds
  float* feat;    // [n][13] closure inputs of the coupling window
  float* ypred;   // [n][8] closure outputs
  double* wnorm;  // [2][n] window density and temperature (0: invalid row)
  unsigned long long* stats;  // rejected, reconstructed, cloned, deleted, learned
  int* fillcnt;               // [DIG_FILL_LAYERS] cells filled per fill layer
  CoupleScalars* scal;
  // synthetic solve (S10): iteration limits, local pseudo-time steps and the
  // Anderson acceleration
  int N_m, aa_m, closed;  // closed: no open boundary face (the solve restores the total mass)
  double eps_m, cfl;
  double* dtl;    // [n] cfl times the cell's CFL-1 pseudo-time step
  double *fp, *Gp;    // [6][n] previous f = g(U) - U and g(U) (Gp holds g(U_k) during an iteration)
  double* Ub;         // [6][n] the best iterate so far
  double *dF, *dG;    // [aa_m][6][n] differences of consecutive f and g(U)
  double* apart;      // [AA_MAX + 1][aab] per-block dot products
  int aab;            // blocks of the Anderson base step (a few per SM, at most one per CPT cells)
  AAState* aa;
  int* rpart;
  int* clone_total;
};

// S9; with ypred non-null the learned closure's outputs replace the HoT.  It
// runs extraction, the reconstruction passes and the first chunk of fill
// layers and leaves in *av the availability array that holds the result.
void launch_couple_s9(const Params& P, const CoupleParams& C, int passes, const float* ypred, int** av,
                      cudaStream_t s);
// fill layers [q0, q1) continuing from availability *av (updated)
void launch_couple_fill(const Params& P, const CoupleParams& C, int q0, int q1, int** av, cudaStream_t s);
// cells still unavailable after the fill layers take the initial state with zero HoT
void launch_couple_unreached(const Params& P, const CoupleParams& C, const int* av, cudaStream_t s);
// closure inputs X[n][13] from sums phi over cnt steps (also fills C.wnorm)
void launch_closure_features(const Params& P, const CoupleParams& C, const double* phi, double cnt, float* X,
                             cudaStream_t s);
// closure targets Y[n_rows][8] from sums phi over cnt steps and input rows X
void launch_closure_targets(const Params& P, const CoupleParams& C, const double* phi, double cnt, const float* X,
                            long long n_rows, float* Y, cudaStream_t s);
// learned closure (dig_mlp.cu); params are the FP32 master parameters
// Y[n][8] = network(X[n][13]) on tcgen05; *status |= 1 if a wait on the
// tensor cores gave up (about a second); hold != 0 withholds the MMAs (a
// test of that path)
void launch_mlp_forward(const float* params, const float* X, long long n, float* Y, int* status, cudaStream_t s,
                        int hold = 0, const float* T = nullptr, double* acc = nullptr);
void launch_mlp_train_step(const float* params, const float* X, const float* T, const int* perm, long long n_total,
                           long long b0, long long nb, float* grad, double* loss, int* status, cudaStream_t s);
void launch_mlp_loss(const float* params, const float* X, const float* T, long long n, int identity, double* acc,
                     int* status, cudaStream_t s);
void launch_adam(float* p, float* m, float* v, float* g, long long t, float lr, float b1, float b2, float eps,
                 cudaStream_t s);
void launch_mlp_init(const Params& P, uint64_t seed, float* params, cudaStream_t s);
// S10: the initial conserved state; `iters` solver iterations (each stops
// early once the solve is done: its state lives on the device), returning
// the number of kernels enqueued (not added to g_launches, so that a stream
// capture can count them); the final primitives
void launch_couple_s10_init(const Params& P, const CoupleParams& C, cudaStream_t s);
long long launch_couple_s10_iters(const Params& P, const CoupleParams& C, int iters, cudaStream_t s);  // kernels enqueued
void launch_couple_s10_final(const Params& P, const CoupleParams& C, cudaStream_t s);
void launch_couple_s11(const Params& P, const CoupleParams& C, const Buf& cur, int N, uint32_t sub, int* cl,
                       cudaStream_t s);
size_t couple_part_count(int n_cells);
size_t couple_apart_count(int n_cells);
// blocks of the Anderson base step: four per SM, at most one per 128 cells
int couple_aa_blocks(int n_cells);

// launchers (dig_kernels.cu)
void launch_init(const Params& P, const Buf& out, int n, cudaStream_t s);
void launch_write(const Params& P, const Buf& out, const double* xs, const float* vs, const float* Is,
                  const int* cells, int n, cudaStream_t s);
void launch_scan(const Params& P, cudaStream_t s);
void launch_scatter(const Params& P, const int* mc, cudaStream_t s);
void launch_cell_pass(const Params& P, const Buf& in, const Buf& out, int pass, int sflags,
                      uint32_t step_coll, uint32_t step_move, double ewma_a, double ewma_b, int tile_cells,
                      int threads,
                      cudaStream_t s);
void launch_inject(const Params& P, const Buf& out, uint32_t step, int wallflux, cudaStream_t s);
void launch_read(const Params& P, const Buf& cur, double* xs, float* vs, float* Is, int* cells,
                 int n, cudaStream_t s);
void launch_moments_ex(const Params& P, const double* phi, double scale, int macro, double* out, double mass,
                       double FN, double kB, cudaStream_t s);
size_t sort_scratch_bytes(long long n, int n_cells);
void launch_sort_by_cell(const int* cell, long long n, int n_cells, int* cell_start, int* order, char* scratch,
                         cudaStream_t s);
int scan_blocks(int n_cells);
// sets the calling thread's message returned by dig_last_error(NULL)
void set_thread_error(const char* msg);
// kernels launched by the library (dig_launch_count); the context-free calls
// may run on several host threads at once
extern std::atomic<long long> g_launches;

}  // namespace dig
