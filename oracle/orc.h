/*
 * orc.h -- plain CPU oracle of the DIG-augmented DSMC hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  The
 * product (paper_2607_08195_gb300, include/dig.h) never calls it and shares
 * no code, header, table or constant generator with it.
 *
 * It follows the paper step by step, single threaded, in the paper's order
 * (DSMC method, Sec. 2.1: move, then collide pairs in the same cell, then
 * sample; statistical treatment, Sec. 3).  Positions and ray-face parameters
 * are FP64, velocities and collision arithmetic FP32, sums FP64.  Compile with
 * -O2 -ffp-contract=off (no -ffast-math): every floating-point decision is
 * then a fixed sequence of IEEE operations.
 *
 * The interface mirrors the shape of the product's C ABI under the prefix
 * orc_ but takes host memory.
 */
#ifndef ORC_H
#define ORC_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_config {
  double mass;      /* molecular mass, kg */
  double d_ref;     /* VHS reference diameter, m */
  double omega;     /* viscosity index */
  double T_ref;     /* reference temperature of d_ref, K */
  double alpha;     /* VSS scattering parameter (1 = VHS) */
  double Z_rot;     /* rotational collision number */
  int32_t rot_dof;  /* 0 (monatomic) or 2 (diatomic) */
  int32_t max_cross;/* face crossings allowed per particle per step */
  double F_N;       /* real molecules per simulation particle */
  double dt;        /* time step, s */
  uint64_t seed;
  double n_init;    /* initial number density, 1/m^3 (informative) */
  double T_init;    /* initial temperature, K */
  double u_init[3]; /* initial drift, m/s */
  double mu_ref;    /* viscosity at T_ref, Pa s */
  double Kn;        /* global Knudsen number */
  double L_ref;     /* reference length, m */
  int32_t n_a;      /* EWMA effective samples (Eq. exponential average) */
  int32_t N_s;      /* DSMC steps per outer coupling cycle */
  int32_t N_m;      /* maximum synthetic-solver iterations */
  int32_t passes;   /* reconstruction passes for rejected cells */
  double eps_m;     /* synthetic-solver residual tolerance */
  double KnD_max;   /* cell Knudsen threshold of the reliability criterion */
  int64_t capacity; /* particle capacity */
  int32_t closure;  /* 1: the learned closure supplies the HoT of the coupling (S12) */
  int32_t recon;    /* reconstruction mean of density and temperatures: 0 arithmetic, 1 logarithmic */
  int32_t local_acc;/* 1: rejected cells enter the local accumulation state (Sec. 3.2) */
  int32_t aa_m;     /* depth of the Anderson acceleration of the synthetic solve (0: plain local steps) */
  double cfl;       /* pseudo-time CFL number of the synthetic solve's local steps (<= 0: 1.5) */
} orc_config;

/* most Anderson-acceleration columns */
#define ORC_AA_MAX 32

typedef struct orc_bc {
  int32_t kind;     /* 0 diffuse wall, 1 specular wall, 2 free-stream inflow, 3 outflow */
  int32_t pad;
  double T;         /* wall or free-stream temperature, K */
  double U[3];      /* wall or free-stream velocity, m/s */
  double n;         /* free-stream number density, 1/m^3 */
} orc_bc;

/* moment selectors for orc_read_moments */
enum { ORC_PHI_INST = 0, ORC_PHI_EWMA = 1, ORC_PHI_WINDOW = 2, ORC_PHI_CUM = 3, ORC_MACRO = 16 };
/* dsmc_step flags */
enum { ORC_EWMA = 1, ORC_WINDOW = 2, ORC_CUMUL = 4, ORC_RECORD_PAIRS = 8 };
/* sample() actions */
enum { ORC_RESET_WINDOW = 1, ORC_RESET_CUMUL = 2, ORC_RESET_EWMA = 4 };
/* counters */
enum { ORC_C_STEPS, ORC_C_CAND, ORC_C_COLL, ORC_C_CROSS, ORC_C_WALL, ORC_C_REMOVED,
       ORC_C_INJECTED, ORC_C_STUCK, ORC_C_LB, ORC_N_COUNTERS };

typedef struct orc_ctx orc_ctx;

orc_ctx* orc_create(const orc_config* cfg);
void orc_destroy(orc_ctx* c);
const char* orc_last_error(orc_ctx* c);

int orc_mesh_load(orc_ctx* c, const double* nodes, int64_t n_nodes, const int32_t* tets,
                  int64_t n_tets, const int32_t* face_tag, const orc_bc* bcs, int32_t n_bcs);
int orc_particles_init(orc_ctx* c, int64_t n);
int orc_write_particles(orc_ctx* c, const double* x, const float* v, const float* Ir,
                        const int32_t* cell, int64_t n);
int orc_read_particles(orc_ctx* c, double* x, float* v, float* Ir, int32_t* cell, int64_t cap,
                       int64_t* n);
int orc_dsmc_step(orc_ctx* c, int32_t n_steps, int32_t flags);
int orc_sample(orc_ctx* c, int32_t action);
int orc_read_moments(orc_ctx* c, int32_t which, double* out, int64_t cap);
int orc_read_pairs(orc_ctx* c, int32_t* cell, int32_t* k, int32_t* i, int32_t* j, uint8_t* acc,
                   int64_t cap, int64_t* n);
int orc_read_counters(orc_ctx* c, int64_t* out, int32_t n);
int orc_cell_state(orc_ctx* c, float* cmax, double* rem, int32_t write);
int orc_wall_flux(orc_ctx* c, double* out, int64_t cap, int64_t* n_bfaces);
int64_t orc_step_index(orc_ctx* c);

/* DIG coupling (Alg. 1: one outer step after N_s DSMC steps) */
typedef struct orc_couple_report {
  int32_t iters;            /* synthetic-solver iterations */
  int32_t n_learned;        /* cells whose HoT came from the learned closure */
  double residual;          /* final residual / first residual */
  int64_t n_rejected;       /* cells failing the cell-Knudsen criterion */
  int64_t n_reconstructed;  /* rejected cells rebuilt from neighbours */
  int64_t n_cloned, n_deleted;
} orc_couple_report;
int orc_couple(orc_ctx* c, orc_couple_report* rep);
/* which: 0 M^{k+1/2} [n][6], 1 HoT [n][12], 2 M^{k+1} [n][6], 3 flags [n], 4 own sampled state [n][6],
 * 5 local accumulation weight [n] (0: moving average) */
int orc_read_couple(orc_ctx* c, int32_t which, double* out, int64_t cap);
/* harness for the pins of the synthetic equations (Sec. 2.2), nondimensional
 * rows per cell: prim [n][6] = rho, u(3), T_t, T_r; grad [n][15] = d(u_x, u_y,
 * u_z, T_t, T_r)/d(x, y, z), component-major within the row (3 q + i);
 * NSF out [n][12] = sigma (xx, yy, zz, xy, xz, yz), q_t (3), q_r (3).
 * orc_synthetic_solve runs the solve from M^{k+1/2} = half with the given HoT
 * [n][12]; src [n][6] (or NULL) is a volume source added to the residual of
 * each conserved variable (rho, rho u, rho E, rho e_r), for a manufactured
 * solution; out [n][6] receives M^{k+1}. */
int orc_gradients(orc_ctx* c, const double* prim, double* grad);
int orc_nsf(orc_ctx* c, const double* prim, const double* grad, double* out);
int orc_synthetic_solve(orc_ctx* c, const double* half, const double* hot, const double* src, double* out,
                        int32_t* iters, double* res);
/* the residual R [n][6] of the conserved variables (rho, rho u, rho E,
 * rho e_r) and the CFL-1 pseudo-time step dtl [n] of the state prim [n][6]
 * with the given HoT [n][12] and source src [n][6] (or NULL) */
int orc_synthetic_residual(orc_ctx* c, const double* prim, const double* hot, const double* src, double* R,
                           double* dtl);
int orc_write_moments(orc_ctx* c, int32_t which, const double* in);
int orc_write_wall_flux(orc_ctx* c, const double* in, int64_t steps);

/* learned closure (S12/S13): MLP 13 -> 64 -> 64 -> 64 -> 8, GELU */
int32_t orc_mlp_nparam(void);
double orc_bf16(double x);
void orc_mlp_init(float* params, uint64_t seed);
int orc_mlp_forward(const float* params, const float* X, int64_t n, int32_t bf16, double* Y);
double orc_mlp_grad(const float* params, const float* X, const float* T, int64_t n, int32_t bf16, double* grad);
void orc_adam(float* params, double* m, double* v, const double* g, int64_t t, double lr, double b1, double b2,
              double eps);
/* closure inputs and targets; a prediction with a component beyond
 * ORC_CLOSURE_YMAX in magnitude (or non-finite) falls back to the sampled HoT */
#define ORC_CLOSURE_YMAX 4.0

/* most fill layers after the reconstruction layers of a coupling */
#define ORC_FILL_LAYERS 1024
int orc_closure_set(orc_ctx* c, const float* params);
int orc_closure_features(orc_ctx* c, int32_t which, float* X);
int orc_closure_targets(orc_ctx* c, int32_t which, const float* X, int64_t n_rows, float* Y);

/* stable counting sort by cell (the paper's per-cell particle buckets):
 * cell[n] in [0, n_cells) or -1 (dropped); writes cell_start[n_cells+1] and
 * order[] = indices of the kept elements sorted by cell, ties by index. */
int orc_sort_by_cell(const int32_t* cell, int64_t n, int32_t n_cells, int32_t* cell_start, int32_t* order);

/* primitives exposed for the pins */
/* unit post-collision directions e[n][3] of the VSS model for relative
 * velocities g[n][3] (non-zero), alpha from the context's config; entity p,
 * sub 0, step 0 of the context's collision-direction random stream */
int orc_vss_directions(orc_ctx* c, const float* g, int64_t n, float* e);
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
float orc_lnf(float x);
float orc_expf(float y);
float orc_powf(float x, float a);
int orc_mesh_info(orc_ctx* c, int32_t* nbr, int8_t* nbr_face, double* normals, double* d,
                  double* vol);
int32_t orc_locate(orc_ctx* c, const double* x, double tol);
int orc_track_one(orc_ctx* c, double* x, float* v, int32_t* cell, int64_t slot, int64_t step);

#ifdef __cplusplus
}
#endif
#endif
