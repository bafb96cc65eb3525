/*
 * dig.h -- C ABI of the GB300 DSMC/DIG library (libdig.so).
 *
 * One simulation context runs the DSMC particle loop of the DIG method
 * (arXiv 2607.08195) on one GPU: move particles face by face through a
 * tetrahedral mesh, sort them by cell, collide pairs in each cell (NTC, VHS,
 * Borgnakke-Larsen), sample cell moments and time-average them.
 *
 * Conventions
 *  - Every function returns int: DIG_OK (0) or a negative DIG_ERR_* code;
 *    dig_last_error() gives the message of the last failure.
 *  - Host pointers are borrowed for the duration of the call only.
 *  - Device memory belongs to the caller: dig_arena_bytes() says how many
 *    bytes one context needs; the caller allocates them (for instance a torch
 *    uint8 tensor), passes the device pointer to dig_bind_arena() and keeps the
 *    allocation alive until dig_destroy().  The library allocates no device
 *    memory of its own.
 *  - All GPU work is queued on the stream given to dig_set_stream() (default:
 *    the legacy default stream).  Functions that return host data wait for the
 *    stream, polling with a time limit (dig_config.wait_timeout_s); a wait that
 *    runs out returns DIG_ERR_TIMEOUT.
 *  - A context is not thread safe.
 *  - Units are SI; rotational energies I_r are stored in kelvin (I_r / k_B).
 */
#ifndef DIG_H
#define DIG_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DIG_OK 0
#define DIG_ERR_ARG (-1)      /* bad argument */
#define DIG_ERR_MESH (-2)     /* mesh rejected (degenerate, non-manifold, untagged boundary) */
#define DIG_ERR_CAPACITY (-3) /* particle capacity or per-cell staging capacity exceeded */
#define DIG_ERR_STUCK (-4)    /* a particle exceeded the face-crossing limit in one step */
#define DIG_ERR_SOLVE (-5)    /* synthetic-equation solve failed (non-finite or diverged) */
#define DIG_ERR_CUDA (-6)     /* CUDA runtime error */
#define DIG_ERR_STATE (-7)    /* call out of order (no mesh, no arena, no particles) */
#define DIG_ERR_TIMEOUT (-8)  /* a host wait on the stream ran out of time */

/* boundary-condition kinds */
#define DIG_BC_DIFFUSE 0
#define DIG_BC_SPECULAR 1
#define DIG_BC_INFLOW 2
#define DIG_BC_OUTFLOW 3

/* dsmc_step flags */
#define DIG_EWMA 1         /* update the exponential moving average (paper Eq. exponential_average_moments;
                              until n_a samples exist it is the plain mean of all samples) */
#define DIG_WINDOW 2       /* add to the coupling-window sums */
#define DIG_CUMUL 4        /* add to the cumulative sums (paper Eq. steady_average_moments) */
#define DIG_RECORD_PAIRS 8 /* debug: record the candidate pairs of the last step */
#define DIG_INST 16        /* keep the instantaneous sums of the last step */
#define DIG_WALLFLUX 32    /* accumulate momentum/energy exchanged with each wall face */
#define DIG_SYNC 64        /* wait for the steps and check the device status before returning */
#define DIG_TIMING 128     /* record CUDA events around every cell-pass launch (see dig_kernel_time) */

/* sample() actions */
#define DIG_RESET_WINDOW 1
#define DIG_RESET_CUMUL 2
#define DIG_RESET_EWMA 4

/* read_moments selectors: raw summation variables (17 doubles per cell) or,
 * with DIG_MACRO added, the 20 derived moments per cell */
#define DIG_PHI_INST 0
#define DIG_PHI_EWMA 1
#define DIG_PHI_WINDOW 2
#define DIG_PHI_CUM 3
#define DIG_MACRO 16
#define DIG_NPHI 17
#define DIG_NMAC 20

/* counters (read_counters) */
#define DIG_C_STEPS 0
#define DIG_C_CAND 1
#define DIG_C_COLL 2
#define DIG_C_CROSS 3
#define DIG_C_WALL 4
#define DIG_C_REMOVED 5
#define DIG_C_INJECTED 6
#define DIG_C_STUCK 7
#define DIG_C_LB 8
#define DIG_N_COUNTERS 9

typedef struct dig_config {
  double mass;       /* molecular mass, kg */
  double d_ref;      /* VHS reference diameter, m */
  double omega;      /* viscosity-temperature index */
  double T_ref;      /* reference temperature of d_ref, K */
  double alpha;      /* VSS scattering parameter, > 0: 1 = VHS (isotropic); otherwise the
                        VSS deflection law (paper Sec. 2.1); also enters P_inelastic */
  double Z_rot;      /* rotational collision number Z_r */
  int32_t rot_dof;   /* rotational degrees of freedom d_r: 0 or 2 */
  int32_t max_cross; /* face crossings allowed per particle per step (<= 0: 4096) */
  double F_N;        /* real molecules per simulation particle (N_eff) */
  double dt;         /* time step, s */
  uint64_t seed;     /* key of every random stream */
  double n_init;     /* initial number density, 1/m^3 (informative) */
  double T_init;     /* temperature of the initial equilibrium state, K */
  double u_init[3];  /* drift velocity of the initial state, m/s */
  double mu_ref;     /* viscosity at T_ref, Pa s */
  double Kn;         /* global Knudsen number (paper Eq. kn_definition) */
  double L_ref;      /* reference length, m */
  int32_t n_a;       /* effective samples of the moving average */
  int32_t N_s;       /* DSMC steps per outer coupling cycle */
  int32_t N_m;       /* maximum synthetic-solver iterations */
  int32_t passes;    /* neighbour-reconstruction passes */
  double eps_m;      /* synthetic-solver residual tolerance */
  double KnD_max;    /* threshold of the cell Knudsen criterion */
  int64_t capacity;  /* particle capacity of the arena */
  double wait_timeout_s; /* time limit of host waits (<= 0: 600 s) */
  int32_t stage_cap;     /* particles per CTA the move kernel's tile of cells aims at: tile = 0.75 stage_cap /
                            mean particles per cell (<= 0: 3072; at most 8192) */
  int32_t tile_cells;    /* cells per CTA of the move kernel, at most 2048 (<= 0: chosen from stage_cap and
                            the load) */
  int32_t cta_threads;   /* threads per CTA of the move kernel: 64, 128 or 256 (<= 0: 256) */
  int32_t closure;       /* 1: dig_couple takes the HoT from the learned closure (see closure_*) */
  int32_t recon;         /* mean of the neighbour reconstruction (Sec. 3.2, every neighbour with the
                            same weight) for density and temperatures: 0 arithmetic, 1 logarithmic
                            (exp of the mean logarithm, the log-mean reconstruction of Sec. 6; the
                            arithmetic mean where a contributing value is not positive); velocity
                            and HoT always arithmetic */
  int32_t local_acc;     /* 1: a cell the filter rejects enters the local accumulation state (Sec. 3.2):
                            its moving average stops forgetting (running mean of every later step,
                            its average so far counting as min(m, n_a) samples) until a coupling
                            accepts it; 0: every cell keeps the moving average */
  int32_t aa_m;          /* synthetic solve (S10): depth of the Anderson acceleration of its pseudo-time
                            iteration, 0..DIG_AA_MAX (0: plain local pseudo-time steps) */
  double cfl;            /* synthetic solve: CFL number of each cell's own pseudo-time step (<= 0: 1.5) */
} dig_config;

/* most Anderson-acceleration columns of the synthetic solve (dig_config.aa_m) */
#define DIG_AA_MAX 32

typedef struct dig_bc {
  int32_t kind;  /* DIG_BC_* */
  int32_t pad;
  double T;      /* wall or free-stream temperature, K */
  double U[3];   /* wall or free-stream velocity, m/s */
  double n;      /* free-stream number density, 1/m^3 (inflow only) */
} dig_bc;

typedef struct dig_ctx dig_ctx;

/* Create a context for one gas and time step.  No GPU work is done.
 * DIG_ERR_ARG unless mass, dt, F_N and alpha are positive, rot_dof is 0 or 2,
 * recon and local_acc are 0 or 1, stage_cap <= 8192 and tile_cells <= 2048
 * (the move kernel's shared memory holds 92 B per cell of its tile). */
int dig_create(const dig_config* cfg, dig_ctx** out);
/* Release the context (the caller then frees its arena). */
int dig_destroy(dig_ctx* ctx);
/* message of the last failure of ctx; with ctx NULL, of the calling thread's
 * last failed context-free call */
const char* dig_last_error(dig_ctx* ctx);
/* Queue all later GPU work on this cudaStream_t (NULL = legacy default stream). */
int dig_set_stream(dig_ctx* ctx, void* cuda_stream);

/*
 * mesh_load -- load a conforming tetrahedral mesh (host arrays, copied).
 * nodes [n_nodes][3] (m); tets [n_tets][4] node indices; face_tag[n_tets][4]:
 * face f of a tet is the face opposite its vertex f; -1 on interior faces,
 * else an index into bcs[n_bcs].  Builds the neighbour table (the paper's
 * face-based tracking, Sec. 4, local mesh package), FP64 face planes, volumes.
 * Errors: DIG_ERR_MESH for zero-volume tets, faces shared by more than two
 * tets, boundary faces without a tag or interior faces with one.
 */
int mesh_load(dig_ctx* ctx, const double* nodes, int64_t n_nodes, const int32_t* tets,
              int64_t n_tets, const int32_t* face_tag, const dig_bc* bcs, int32_t n_bcs);

/* Device bytes the context needs for the loaded mesh and cfg.capacity particles. */
int dig_arena_bytes(dig_ctx* ctx, int64_t* bytes);
/* Bind caller-owned device memory (256-byte aligned, >= dig_arena_bytes) and
 * upload the mesh tables.  The memory must outlive the context. */
int dig_bind_arena(dig_ctx* ctx, void* device_ptr, int64_t bytes);

/*
 * particles_init -- n particles in the uniform equilibrium state of cfg
 * (paper Sec. 5.1: rho, u = u_init, T_t = T_r = T_init), cell by inverse CDF of
 * the cell volumes, uniform position in the tet, Maxwellian velocity; then the
 * particles are sorted by cell.  DIG_ERR_CAPACITY if n > capacity.
 */
int particles_init(dig_ctx* ctx, int64_t n);

/* write_particles / read_particles -- HOST arrays: x [n][3] f64, v [n][3] f32,
 * Ir [n] f32 (may be NULL; ignored and read back as 0 for a monatomic gas),
 * cell [n] i32.  write sorts by cell, keeping the
 * given order inside each cell.  read returns the particles sorted by cell
 * (the order the next collision step uses) and their count in *n; with
 * cap < count nothing is copied and DIG_ERR_CAPACITY is returned. */
int write_particles(dig_ctx* ctx, const double* x, const float* v, const float* Ir,
                    const int32_t* cell, int64_t n);
int read_particles(dig_ctx* ctx, double* x, float* v, float* Ir, int32_t* cell, int64_t cap,
                   int64_t* n);

/*
 * dsmc_step -- advance n_steps DSMC time steps (paper Sec. 2.1; Alg. 1,
 * "perform N_s standard DSMC time steps"): move with wall interaction and
 * removal at open boundaries, sort by cell, NTC collisions, sampling; flags
 * select which time averages are updated (DIG_EWMA, DIG_WINDOW, DIG_CUMUL,
 * DIG_INST, DIG_WALLFLUX, DIG_RECORD_PAIRS).  Asynchronous unless DIG_SYNC is
 * given; device-side errors (capacity, stuck particles) are then reported by
 * the next call that waits.
 */
int dsmc_step(dig_ctx* ctx, int32_t n_steps, int32_t flags);

/* sample -- reset time averages (DIG_RESET_WINDOW / _CUMUL / _EWMA bits). */
int sample(dig_ctx* ctx, int32_t action);

/*
 * read_moments -- copy per-cell sums to host out[n_tets][17] (which = DIG_PHI_*)
 * or derived moments out[n_tets][20] (which | DIG_MACRO): mean N, rho, u(3),
 * T_t, T_r, T, sigma (xx,yy,zz,xy,xz,yz), q_t(3), q_r(3), paper
 * Eq. dsmc_temperatures in SI units.  Window and cumulative sums are divided
 * by their step counts before the moments are derived.
 */
int read_moments(dig_ctx* ctx, int32_t which, double* host_out, int64_t cap);

/* debug: candidate pairs of the last step run with DIG_RECORD_PAIRS, sorted by
 * (cell, k): cell, candidate index k, first i and second j index inside the
 * cell (sorted order), accepted flag.  With any output pointer NULL only the
 * count is returned in *n. */
int read_pairs(dig_ctx* ctx, int32_t* cell, int32_t* k, int32_t* i, int32_t* j, uint8_t* acc,
               int64_t cap, int64_t* n);
int read_counters(dig_ctx* ctx, int64_t* out, int32_t n);
/* per-cell collision state (sigma c_r)_max (f32) and NTC remainder (f64), host arrays */
int dig_cell_state(dig_ctx* ctx, float* cmax, double* rem, int32_t write);
/* per boundary face (in (tet, face) order): hits, momentum (3) and energy given
 * to the wall, out[n_bfaces][5]; with out NULL only *n_bfaces is set. */
int dig_wall_flux(dig_ctx* ctx, double* out, int64_t cap, int64_t* n_bfaces);
/* surface quantities of every boundary face (in (tet, face) order) from the
 * wall-flux sums of the steps run with DIG_WALLFLUX since the last coupling
 * (or dig_write_wall_flux): out[n_bfaces][6] = number flux of molecules
 * hitting the face (1/(m^2 s)), pressure (normal momentum flux into the wall,
 * Pa), shear stress (the tangential momentum flux vector, 3 components, Pa)
 * and heat flux into the wall (W/m^2), per unit face area and time.  With out
 * NULL only *n_bfaces is set; DIG_ERR_STATE if no step was sampled. */
int dig_surface(dig_ctx* ctx, double* out, int64_t cap, int64_t* n_bfaces);
int dig_particle_count(dig_ctx* ctx, int64_t* n);
/* wait for all queued work; returns the first device-side error, if any */
int dig_synchronize(dig_ctx* ctx);
/* number of kernels the library launched (all contexts of the process) */
int dig_launch_count(dig_ctx* ctx, int64_t* n);
/* Sum of the device times of the cell-pass launches recorded with DIG_TIMING
 * since the last call (CUDA events on the context's stream; waits for them),
 * and how many launches they were.  Resets the record. */
int dig_kernel_time(dig_ctx* ctx, double* total_ms, int64_t* launches);

/*
 * DIG coupling -- one outer step of the paper's Alg. 1 after N_s DSMC steps:
 * from the moving-average sums, M^{k+1/2} and HoT = sampled stress / heat
 * flux minus their NSF values (Sec. 3.1, Eq. hot_extraction), the cell
 * Knudsen criterion Kn_Delta <= KnD_max (Sec. 3.2; a cell whose moving
 * average holds fewer than two particles on average is rejected too) with `passes` layers of
 * equal-weight neighbour reconstruction (rejected cells beyond them are
 * filled the same way, layer by layer, up to 64 more layers, and are not
 * recalibrated), the steady synthetic equations
 * (Eq. macro with Eq. synthetic_closure) solved for M^{k+1} (at most N_m
 * iterations or residual below eps_m of its first value; pseudo-time
 * iteration with each cell's own step at CFL cfg.cfl, Anderson acceleration
 * of depth cfg.aa_m, and, without open boundaries, a scaling that keeps the
 * total mass of M^{k+1/2}), and the particles
 * of accepted cells recalibrated to M^{k+1} (velocities shifted and scaled,
 * rotational energies scaled, particles cloned or deleted with the density
 * ratio against the density of the particles the cell holds).  Diffuse walls
 * close the synthetic equations as isothermal no-slip walls (the wall velocity
 * and temperature enter the gradients; the wall face carries the cell's
 * pressure, total stress and heat flux and the flux scheme's dissipation
 * against the mirrored state), specular
 * walls as slip walls (pressure only); the wall fluxes sampled with
 * DIG_WALLFLUX remain a DSMC output (dig_wall_flux).  With
 * cfg.closure = 1 and closure parameters set, the translational HoT (sigma,
 * q_t) of each cell comes from the learned closure evaluated on the coupling
 * window's sums (DIG_WINDOW; see closure_features), except for cells whose
 * window is empty or whose prediction is non-finite or has a component beyond
 * DIG_CLOSURE_YMAX: they keep the sampled HoT.  Synchronous;
 * DIG_ERR_SOLVE if the solve produced a non-finite or non-positive state (the
 * particles are then left unchanged).
 */
typedef struct dig_couple_report {
  int32_t iters;            /* synthetic-solver iterations */
  int32_t n_learned;        /* cells whose HoT came from the learned closure */
  double residual;          /* final residual relative to the first one */
  int64_t n_rejected;       /* cells failing the cell-Knudsen criterion */
  int64_t n_reconstructed;  /* rejected cells rebuilt from their neighbours */
  int64_t n_cloned, n_deleted;
} dig_couple_report;
int dig_couple(dig_ctx* ctx, dig_couple_report* out);
/* coupling fields of the last dig_couple, host out[n_tets][k], nondimensional
 * (density / (m n_init), velocity / sqrt(k T_init / m), temperature / T_init):
 * which 0 = M^{k+1/2} fed to the solver (rho, u(3), T_t, T_r; k = 6),
 * 1 = HoT (sigma xx,yy,zz,xy,xz,yz, q_t(3), q_r(3); k = 12), 2 = M^{k+1}
 * (k = 6), 3 = cell flags (1 accepted, 2 reconstructed, 3 filled beyond the
 * reconstruction layers, 0 none of these; k = 1),
 * 4 = each cell's own sampled state (k = 6), 5 = each cell's local
 * accumulation weight (samples its moving average stands for in the local
 * accumulation state, 0 outside it; k = 1, current value) */
int dig_read_couple(dig_ctx* ctx, int32_t which, double* host_out, int64_t cap);
/* overwrite summation variables (which = DIG_PHI_*) from host in[n_tets][17] */
int dig_write_moments(dig_ctx* ctx, int32_t which, const double* host_in);
/* overwrite the per-wall-face sums in[n_bfaces][5] (hits, momentum, energy
 * given to the wall) and the number of DSMC steps they cover */
int dig_write_wall_flux(dig_ctx* ctx, const double* host_in, int64_t steps);

/*
 * Checkpoint / resume.  A checkpoint is the context's whole device state (the
 * bound arena: particles, cell tables, summation variables, remainders, the
 * collision maxima, coupling fields, closure parameters and Adam moments) and
 * its host counters (step, sample counts, coupling count, particle count), so
 * that a run resumed from it continues bit for bit: every random number is
 * keyed by counters the checkpoint holds.
 * dig_checkpoint_bytes: the size in bytes.  dig_save: write it to host memory
 * host_out (cap >= that size; DIG_ERR_CAPACITY otherwise).  dig_load: restore
 * it into a context created with the same configuration and mesh and bound to
 * an arena of the same size (DIG_ERR_STATE otherwise; DIG_ERR_ARG for a buffer
 * that is not a checkpoint or is truncated).  Both wait for the stream and
 * need a bound arena (DIG_ERR_STATE).  The caller owns host_out / host_in.
 */
int dig_checkpoint_bytes(dig_ctx* ctx, int64_t* bytes);
int dig_save(dig_ctx* ctx, void* host_out, int64_t cap);
int dig_load(dig_ctx* ctx, const void* host_in, int64_t size);

/*
 * Learned closure (not in the paper; the DIG HoT from a per-cell network):
 * an MLP 13 -> 64 -> 64 -> 64 -> 8 with GELU (z/2 (1 + erf(z / sqrt 2))) on
 * the hidden layers, BF16 weights and activations, FP32 accumulation on the
 * tcgen05 tensor cores (accumulators in tensor memory, 128 rows per tile) in
 * the forward pass, the loss and the training step.  Every wait on the
 * tensor cores gives up after about a second; the calls below then return
 * DIG_ERR_TIMEOUT.  Parameters (FP32 master copy, [out][in] per layer):
 * W1[64][13] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[8][64] b4[8],
 * DIG_MLP_NPARAM floats; the biases are not rounded to BF16.
 * Inputs (closure_features), per cell, nondimensional as in dig_read_couple:
 * rho, u(3), T_t, the traceless HoT stress (xx, yy, xy, xz, yz) / (rho T_t)
 * and translational HoT heat flux (3) / (rho T_t^{3/2}) -- in SI, sigma over
 * rho k T / m and q over rho (k T / m)^{3/2}.  Outputs: the same eight HoT
 * components, normalised the same way by the input's rho and T_t.
 * Device arrays (X, Y, perm) are the caller's, read or written on the
 * context's stream; rows are contiguous (X [n][13], Y [n][8], f32).
 */
#define DIG_MLP_NIN 13
#define DIG_MLP_NOUT 8
#define DIG_MLP_NPARAM 9736
#define DIG_CLOSURE_YMAX 4.0
/* He-normal weights (std sqrt(2 / fan_in)) from the seed's MLP_INIT random
 * stream, zero biases; resets the Adam state.  Needs a bound arena. */
int closure_init(dig_ctx* ctx, uint64_t seed);
/* copy parameters from / to HOST params[n], n = DIG_MLP_NPARAM (else
 * DIG_ERR_ARG); set resets the Adam state */
int closure_set(dig_ctx* ctx, const float* params, int64_t n);
int closure_get(dig_ctx* ctx, float* params, int64_t n);
/* X[n_tets][13] (DEVICE): the inputs of every cell from the sums `which`
 * (DIG_PHI_*; window and cumulative sums are averaged over their steps); a
 * cell without particles gets a zero row.  Asynchronous. */
int closure_features(dig_ctx* ctx, int32_t which, float* X);
/* training targets Y[n_rows][8] (DEVICE): the HoT of the sums `which` (the
 * long-time average) of cell r mod n_tets, normalised by the density X[r][0]
 * and temperature X[r][4] of input row r (X: n_rows stacked closure_features
 * outputs); zero for rows with zero density or temperature or an empty cell.
 * Asynchronous. */
int closure_targets(dig_ctx* ctx, int32_t which, const float* X, int64_t n_rows, float* Y);
/* Y[n][8] = network(X[n][13]) (DEVICE), on the tcgen05 tensor cores (BF16
 * operands, FP32 accumulators in tensor memory, 128 rows per tile).
 * Synchronous; DIG_ERR_TIMEOUT if a wait on the tensor cores gave up (about
 * a second). */
int closure_forward(dig_ctx* ctx, const float* X, int64_t n, float* Y);
/* Test of the failure path of the closure's tensor-core forward: runs it on
 * up to 128 rows of the context's own buffers with its MMAs withheld, so that
 * its first mbarrier wait gives up after about a second (a flag that nothing
 * sets); the kernel then frees its tensor memory and returns.  Returns what
 * closure_forward returns in that case, DIG_ERR_TIMEOUT; the context stays
 * usable.  Synchronous (about two seconds). */
int dig_test_forward_timeout(dig_ctx* ctx);
/* mean-square error L = 1/(8 n) sum (pred - Y)^2 over n rows (DEVICE X, Y):
 * pred = network(X), or with identity = 1 the inputs' own HoT X[:, 5:13]
 * (the closure without the network).  Synchronous; DIG_ERR_TIMEOUT as above. */
int closure_loss(dig_ctx* ctx, const float* X, const float* Y, int64_t n, int32_t identity, double* loss);
/* gradient of L over all n rows with respect to every parameter, to HOST
 * grad[DIG_MLP_NPARAM] (FP32); *loss = L.  No update.  Synchronous;
 * DIG_ERR_TIMEOUT as above. */
int closure_grad(dig_ctx* ctx, const float* X, const float* Y, int64_t n, float* grad, double* loss);
typedef struct dig_train_cfg {
  int32_t epochs;        /* passes over the rows (>= 1) */
  int32_t batch;         /* rows per Adam step (>= 1) */
  double lr, beta1, beta2, eps; /* Adam (Kingma and Ba 2015) */
  const int32_t* perm;   /* DEVICE [epochs][n]: row order of each epoch, a
                            permutation of 0..n-1; NULL: rows in order */
} dig_train_cfg;
/* Adam on the mean-square error over mini-batches of the rows X[n][13] ->
 * Y[n][8] (DEVICE); loss[epochs] (HOST) receives each epoch's mean training
 * loss.  The Adam step count carries over between calls.  DIG_ERR_ARG for a
 * bad cfg or a perm entry outside [0, n) (found on the device: the epoch's
 * rows with such entries are skipped); DIG_ERR_TIMEOUT as above.  Synchronous. */
int closure_train(dig_ctx* ctx, const dig_train_cfg* cfg, const float* X, const float* Y, int64_t n,
                  double* loss);

/*
 * dig_sort_by_cell -- stable counting sort by cell, the paper's per-cell
 * particle buckets (Sec. 4, Listing 2: one particle bucket per owned cell) as
 * a standalone op on DEVICE arrays, queued on `stream` (a cudaStream_t; NULL =
 * legacy default stream) and asynchronous.
 *   cell[n]       (device, int32) cell of each element; entries outside
 *                 [0, n_cells) are dropped (-1 marks a removed particle)
 *   cell_start    (device, int32 [n_cells+1]) output: start of each cell's
 *                 segment in order[], cell_start[n_cells] = kept count
 *   order         (device, int32 [n]) output: indices of the kept elements,
 *                 sorted by cell, ties by index
 *   scratch       (device, 256-byte aligned, >= dig_sort_scratch_bytes(n,
 *                 n_cells) bytes) caller-owned working memory; its contents
 *                 on entry do not matter
 * Errors (host checks only, nothing launched): DIG_ERR_ARG for bad sizes or
 * pointers, DIG_ERR_CAPACITY for a too small scratch; the message is
 * dig_last_error(NULL) of the calling thread.  n < 2^31.
 */
int dig_sort_scratch_bytes(int64_t n, int32_t n_cells, int64_t* bytes);
int dig_sort_by_cell(const int32_t* cell, int64_t n, int32_t n_cells, int32_t* cell_start, int32_t* order,
                     void* scratch, int64_t scratch_bytes, void* stream);

/*
 * dig_sort_by_cell_noalloc -- the same sort as dig_sort_by_cell, for callers
 * that cannot allocate device memory (their device memory is owned and
 * planned by a host framework or a fixed budget, or cudaMalloc's implicit
 * synchronisation is not allowed where they run).  The paper has no
 * counterpart: this is a deployment variant of the bucket sort.
 * The caller still passes the device inputs and outputs (as for
 * dig_sort_by_cell); the working memory is a fixed array of
 * DIG_NOALLOC_SCRATCH_BYTES inside the library, present on every GPU that
 * loads the library until the process exits.  Limits: n <= DIG_NOALLOC_MAX_N,
 * n_cells <= DIG_NOALLOC_MAX_CELLS; larger sizes return DIG_ERR_CAPACITY
 * (message in dig_last_error(NULL)) without launching anything.  The call
 * allocates nothing.  All calls share the array: calls whose GPU work overlaps
 * (other streams, other threads) race and give wrong results.  Every call
 * looks up the array's device address (cudaGetSymbolAddress) for the device
 * current at the call, so it stays right after the context is destroyed and
 * made again; the first call on a device loads the library's module there:
 * make it before capturing any stream on that device.
 */
#define DIG_NOALLOC_MAX_N 4194304
#define DIG_NOALLOC_MAX_CELLS 1048576
#define DIG_NOALLOC_SCRATCH_BYTES 25167104
int dig_sort_by_cell_noalloc(const int32_t* cell, int64_t n, int32_t n_cells, int32_t* cell_start, int32_t* order,
                             void* stream);

#ifdef __cplusplus
}
#endif
#endif
