/*
 * slim.h - C ABI of the GB300 (sm_103a) implementation of the 3D discontinuous
 * Galerkin ocean-model hot path of arXiv 2605.16082 (SLIM): the element-wise
 * residual of the extruded prismatic P1xP1 mesh, the depth integration that
 * couples the 3D and 2D modes, and the column-wise implicit vertical solves.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Mesh.  n_tri counter-clockwise triangles, each extruded into a column of
 *   n_layers[t] prisms (Sec. 1, Sec. 2.1).  Prism p = col_off[t] + k is layer k
 *   (k = 0 at the surface) of column t, col_off the exclusive prefix sum of
 *   n_layers.  P = total prisms.  Edge e of a triangle joins its vertices e and
 *   (e+1) % 3.
 * 3D nodal fields (6P values): node (c, a, p) at index (c*3 + a)*P + p, c = 0 the
 *   top node and c = 1 the bottom node of prism p, a the triangle vertex.  The
 *   six node planes stream contiguously down every column (the structure-of-
 *   arrays order of Sec. 2.1, field -> node -> column -> layer).
 * 2D nodal fields (3*n_tri values): vertex a of triangle t at index a*n_tri + t.
 * Host pointers are read (or written) during the call only and stay owned by
 *   the caller.  Device pointers ("_dev") are caller-owned, contiguous, and must
 *   hold the stated number of elements of the state's compute type: double for
 *   SLIM_FP64, float for SLIM_MIXED (except where a signature says double).
 * Streams are cudaStream_t passed as void* (0 = legacy default stream).  Work is
 *   enqueued asynchronously unless stated otherwise.
 * Errors: every call returns slim_status; nothing is thrown across the ABI.
 *   slim_last_error() gives a human-readable message for the calling thread.
 *   Device-side conditions (non-finite values, exhausted waits) are latched in a
 *   device flag and reported by slim_state_check().
 * Thread safety: calls on different states are independent; calls on one state
 *   must not overlap on the host.
 */
#ifndef SLIM_H
#define SLIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct slim_mesh slim_mesh;
typedef struct slim_state slim_state;

typedef enum {
  SLIM_OK = 0,
  SLIM_ERR_ARG = 1,        /* invalid argument (null pointer, size, enum)          */
  SLIM_ERR_MESH = 2,       /* inconsistent mesh (orientation, adjacency, layers)   */
  SLIM_ERR_CUDA = 3,       /* a CUDA runtime call failed                            */
  SLIM_ERR_OOM = 4,        /* device allocation failed                              */
  SLIM_ERR_NONFINITE = 5,  /* a kernel produced NaN or Inf                          */
  SLIM_ERR_CFL = 6,        /* time step above the stability estimate                */
  SLIM_ERR_BOUNDS = 7,     /* an index left its range                               */
  SLIM_ERR_TIMEOUT = 8,    /* a bounded device wait gave up                         */
  SLIM_ERR_UNSUPPORTED = 9 /* combination not available (scheme, precision, field)  */
} slim_status;

typedef enum { SLIM_FP64 = 0, SLIM_MIXED = 1 } slim_precision;

/* Time scheme of slim_step. */
typedef enum {
  /* transport frozen over the step, SSP-RK3 explicit horizontal terms with an
     implicit vertical solve in every stage (tracer workload) */
  SLIM_SCHEME_TRACER = 0,
  /* two-stage split-IMEX internal step with subcycled 2D external mode
     (Sec. 2, Eqs. 11-14) */
  SLIM_SCHEME_SPLIT = 1
} slim_scheme;

/* Field identifiers for upload / download. */
enum {
  SLIM_FIELD_T = 0,    /* 3D temperature (or the passive tracer)                      */
  SLIM_FIELD_S = 1,    /* 3D salinity                                                 */
  SLIM_FIELD_U = 2,    /* 3D horizontal velocity, x component [m/s]                   */
  SLIM_FIELD_V = 3,    /* 3D horizontal velocity, y component                         */
  SLIM_FIELD_W = 4,    /* 3D vertex-weighted vertical flux of the last continuity solve */
  SLIM_FIELD_R_X = 5,  /* 3D horizontal baroclinic pressure gradient r, x (Eq. 8)     */
  SLIM_FIELD_R_Y = 6,
  SLIM_FIELD_T_EXT = 7, /* open-boundary exterior profile of T (upload only resets it) */
  SLIM_FIELD_S_EXT = 8, /* open-boundary exterior profile of S                          */
  SLIM_FIELD_ETA = 16, /* 2D elevation [m]                                            */
  SLIM_FIELD_QX = 17,  /* 2D depth-integrated transport [m^2/s]                       */
  SLIM_FIELD_QY = 18,
  SLIM_FIELD_ETA_NEXT = 19, /* 2D elevation at the end of the last continuity solve  */
  SLIM_FIELD_QBAR_X = 20,   /* 2D time-averaged transport of the last external run    */
  SLIM_FIELD_QBAR_Y = 21,
  SLIM_FIELD_S3_X = 22,     /* 2D column sum of the 3D horizontal momentum terms (last stage) */
  SLIM_FIELD_S3_Y = 23,
  SLIM_FIELD_F2D_X = 24,    /* 2D momentum forcing F2D of the last stage (Sec. 2.2)          */
  SLIM_FIELD_F2D_Y = 25,
  /* Open-boundary forcing of the split scheme (read at open-boundary nodes only;
   * used when slim_params.forcing = 1): exterior velocity at time forcing_t_a
   * (U_EXT, V_EXT) and at forcing_t_b (U_EXT_B, V_EXT_B), exterior tracers at
   * forcing_t_b (T_EXT_B, S_EXT_B; those at forcing_t_a are T_EXT, S_EXT).  An
   * upload of a time-a field also sets its time-b field (steady forcing needs one
   * upload); uploading T or S sets both exterior tracer levels. */
  SLIM_FIELD_U_EXT = 26,
  SLIM_FIELD_V_EXT = 27,
  SLIM_FIELD_U_EXT_B = 28,
  SLIM_FIELD_V_EXT_B = 29,
  SLIM_FIELD_T_EXT_B = 30,
  SLIM_FIELD_S_EXT_B = 31
};

typedef struct slim_params {
  double g;            /* gravity [m/s^2]                                  */
  double rho0;         /* reference density [kg/m^3]                       */
  double coriolis_f;   /* Coriolis parameter [1/s]                         */
  double eos_alpha;    /* linear EOS thermal expansion [1/K]               */
  double eos_beta;     /* linear EOS haline contraction [1/psu]            */
  double eos_T0, eos_S0;
  double kappa_v;      /* vertical tracer diffusivity [m^2/s]              */
  double nu_v;         /* vertical viscosity [m^2/s]                       */
  double kappa_h;      /* horizontal tracer diffusivity [m^2/s]            */
  double nu_h;         /* horizontal viscosity [m^2/s]                     */
  double drag_cd;      /* quadratic bottom drag coefficient                */
  double flux_top;     /* prescribed kappa dT/dz at the surface (tracer)   */
  double flux_bot;     /* prescribed kappa dT/dz at the bed (tracer)       */
  double penalty_v;    /* vertical SIPG penalty factor (sigma = p kappa / min dz) */
  double penalty_h;    /* horizontal SIPG penalty factor (sigma = p nu / r_in)    */
  double tide_amp;     /* open-boundary elevation amplitude [m]            */
  double tide_period;  /* open-boundary elevation period [s]               */
  int scheme;          /* slim_scheme                                      */
  int n_sub;           /* external-mode steps per internal step (split)    */
  int tile_prisms;     /* prisms per thread block (0 = default 256)        */
  int check_every;     /* slim_step checks the device error flag every n steps (0 = never) */
  int blocks_per_sm;   /* register budget of the heavy split kernels of the mixed form:
                          2, 3 or 4 resident blocks of 256 threads per SM (0 = default
                          4; 3 is taken as 2 with 512-prism tiles; the FP64 form
                          always uses 2)                                          */
  int use_graph;       /* 1: slim_step replays one CUDA graph of the whole step (captured
                          on the first call and again whenever dt changes; only the
                          step's start time is updated between replays); 0: launches
                          every kernel.  Profiling (slim_profile_begin) uses launches. */
  int persistent_2d;   /* 1: the mixed form's 2D external run of a stage is one
                          cooperative launch over all subcycles with a grid barrier
                          between stages (bounded wait: SLIM_ERR_TIMEOUT via the error
                          flag); 0: one launch per stage.  Same results bit for bit. */
  double forcing_t_a;  /* times of the two open-boundary forcing states (forcing_t_b >  */
  double forcing_t_b;  /* forcing_t_a); the data are linear in time between and beyond */
  int forcing;         /* 1: split scheme with prescribed exterior velocity and tracers at
                          open boundaries, interpolated in time inside the kernels: the
                          2D mode takes the exterior transport Q_ext(t) (the column sum
                          of (dz_rest/2) u_ext) at every stage time, the 3D open faces
                          the exterior transport and state at the middle of the stage's
                          2D run plus their layer share of the averaged 2D face flux
                          (Sec. 3 forcing data, Sec. 2.5 consistency); 0: zero exterior
                          transport in both (a characteristic condition around the tide
                          elevation) and static exterior tracer profiles. */
  int vertical;        /* column system of the implicit vertical terms (Sec. 2.4):
                          0: lumped onto the vertex columns, one 2x2-block tridiagonal
                             system per vertex column (both schemes);
                          1: coupled, the consistent-mass system with one 6x6 block per
                             prism (the paper's fully-assembled column solver): mass,
                             vertical advection and diffusion keep the consistent M_h,
                             the continuity solves the printed D_vd with M_h blocks for
                             the nodal vertical flux (SLIM_FIELD_W then holds Omega) and
                             the elevation takes the consistent 2D mass.  Tracer scheme
                             only (SLIM_ERR_UNSUPPORTED with the split scheme); its
                             shared-memory tile must fit 227 KB (FP64 with 512-prism
                             tiles does not: SLIM_ERR_UNSUPPORTED). */
} slim_params;

/* Fill *p with the defaults: g 9.81, rho0 1025, f 1e-4, alpha 2e-4, beta 7.6e-4,
   T0 10, S0 35, kappa_v = nu_v = 1e-3, kappa_h = nu_h = 0, Cd 2.5e-3, no boundary
   fluxes, penalty_v 4, penalty_h 6, tide 1 m / 44712 s, SLIM_SCHEME_TRACER,
   n_sub 20, tile 256, check_every 0, blocks_per_sm 0, use_graph 1, persistent_2d 1,
   forcing 0 (forcing_t_a 0, forcing_t_b 1), vertical 0.  Returns
   SLIM_ERR_ARG for a null pointer. */
slim_status slim_params_default(slim_params* p);

const char* slim_status_string(slim_status s);
/* Message of the last failing call on this thread ("" if none). */
const char* slim_last_error(void);

/* ---------------------------------------------------------------------------
 * Mesh (Sec. 1 "prismatic mesh made by extruding the 2D mesh"; Sec. 2.1)
 *
 * xy        [2*n_vert]  vertex coordinates, x0 y0 x1 y1 ...
 * tri       [3*n_tri]   counter-clockwise vertex indices
 * h_tri     [3*n_tri]   rest water depth (> 0) at each triangle vertex, tri-major
 *                       (t*3 + a); equal across triangles for sigma layers, a
 *                       staircase depth for z-levels
 * n_layers  [n_tri]     layers of each column, 1..SLIM_MAX_LAYERS
 * levels    [n_levels]  rest interface depths 0 = z_0 > z_1 > ... for z-level
 *                       layering (interface k of a column with N layers sits at
 *                       levels[k] for k < N and at -h at the bed), or NULL for
 *                       uniform sigma layers
 * bnd       [3*n_tri]   per edge (t*3 + e): 0 interior, 1 wall, 2 open boundary
 *
 * Builds the edge adjacency, the per-triangle geometry and the thread-block
 * tiling on the host and copies them to the current CUDA device.  Errors:
 * SLIM_ERR_ARG (null/size), SLIM_ERR_MESH (clockwise triangle, edge shared by
 * more than two triangles, interior edge tagged as boundary or vice versa),
 * SLIM_ERR_OOM / SLIM_ERR_CUDA.  On error *out is NULL.
 * ------------------------------------------------------------------------- */
#define SLIM_MAX_LAYERS 128
slim_status slim_mesh_create(const double* xy, int n_vert, const int* tri, int n_tri,
                             const double* h_tri, const int* n_layers, const double* levels,
                             int n_levels, const signed char* bnd, int tile_prisms,
                             slim_mesh** out);
void slim_mesh_destroy(slim_mesh* m);
/* slim_mesh_create_part: a partition's mesh for the partitioned step (Sec. 3,
 * "Multi-GPU": horizontal partitions with one layer of ghost triangles).  Same
 * arguments as slim_mesh_create plus
 *   tri_class [n_tri]  non-decreasing: 0 an owned triangle with a ghost neighbour,
 *                      1 an owned triangle without, 2 a ghost triangle (a copy of
 *                      another partition's triangle; its edges that leave the
 *                      partition are walls)
 * Thread-block tiles never mix classes, so the kernels can run over the boundary
 * tiles, the interior tiles or both.  Errors as slim_mesh_create, SLIM_ERR_ARG for
 * a missing or unordered tri_class. */
slim_status slim_mesh_create_part(const double* xy, int n_vert, const int* tri, int n_tri,
                                  const double* h_tri, const int* n_layers, const double* levels,
                                  int n_levels, const signed char* bnd, int tile_prisms,
                                  const signed char* tri_class, slim_mesh** out);
/* Sizes of a mesh (any pointer may be NULL). */
slim_status slim_mesh_info(const slim_mesh* m, int64_t* n_prisms, int* n_tri, int* max_layers,
                           int* n_tiles);

/* ---------------------------------------------------------------------------
 * State: device buffers of all fields of one simulation, in the precision's
 * compute type (SLIM_MIXED: 3D fields in float, 2D elevation, transport and
 * their time averages in double).  Fields start at zero.  The mesh must outlive
 * the state.  Errors: SLIM_ERR_ARG, SLIM_ERR_OOM, SLIM_ERR_CUDA.
 * ------------------------------------------------------------------------- */
slim_status slim_state_alloc(const slim_mesh* m, slim_precision prec, const slim_params* par,
                             slim_state** out);
void slim_state_free(slim_state* s);
/* Replace the parameters (same scheme); takes effect at the next call. */
slim_status slim_state_set_params(slim_state* s, const slim_params* par);
/* Copy a field from host doubles (6P or 3*n_tri values, layout above) into the
   state, converting to the compute type; enqueued on the stream, the host
   buffer must stay valid until the stream reaches the copy (synchronous for
   pageable memory).  Uploading T or S also sets the open-boundary exterior
   profile of that tracer. */
slim_status slim_state_upload(slim_state* s, int field, const double* host, void* stream);
/* Copy a field to host doubles; synchronises the stream. */
slim_status slim_state_download(slim_state* s, int field, double* host, void* stream);
/* Device address and element size (4 or 8) of a field buffer of the state. */
slim_status slim_state_field_ptr(slim_state* s, int field, void** dev, int* elem_size);
/* Read and clear the device error flag (synchronises the stream). */
slim_status slim_state_check(slim_state* s, void* stream);

/* ---------------------------------------------------------------------------
 * Hot-path operations
 * ------------------------------------------------------------------------- */

/* slim_rhs3d: horizontal residual of a 3D field at the state's elevation, with the
 * layer transport q = (dz/2) u of the state's velocity.
 * field SLIM_FIELD_T or _S: the tracer residual (Eq. 6, horizontal part)
 *   out[c,a,p] = int_K q T . grad(phi_a) psi_c  -  sum_faces int phi_a psi_c (q.n)^ T^
 *   face transport averaged over both sides, T^ upwind at the face quadrature
 *   points, no flux through walls.
 * field SLIM_FIELD_U or _V (SLIM_SCHEME_SPLIT, forcing 0): one component of the
 *   3D horizontal momentum term F_3D^h of Sec. 2.2 (Eq. 11): upwind advection
 *   -div(q u), horizontal SIPG viscosity nu_h, Coriolis, the baroclinic pressure
 *   gradient -r/rho0 (integrated exactly) and the quadratic bed drag, open faces
 *   with the own transport and zero-gradient velocity (the prediction of the
 *   split step).  r is recomputed first from the state's T, S (as slim_hpg:
 *   SLIM_FIELD_R_X/Y are overwritten), and the FP64 column sums of both components
 *   (the 3D-to-2D coupling S3) are left in SLIM_FIELD_S3_X / _S3_Y.
 * out_dev: 6P elements of the compute type. */
slim_status slim_rhs3d(slim_state* s, int field, void* out_dev, void* stream);

/* slim_continuity: with the transport frozen at the state's elevation eta,
 * (i) the depth-integrated continuity (Eq. 2): (J_h/6)(eta' - eta)/dt equals the
 *     column sum of the horizontal residual of T = 1, written to SLIM_FIELD_ETA_NEXT
 *     in double (FP64 in both precisions);
 * (ii) the vertical flux of every vertex column from the bottom-up column system
 *     of Eq. 17 (printed D_vd pattern), written to SLIM_FIELD_W.
 * With slim_params.vertical = 1 the 2D mass is the consistent M_h (M_h (eta' -
 * eta)/dt = the column sum) and (ii) solves D_vd (x) M_h for the nodal flux Omega.
 * The state's eta is not modified. */
slim_status slim_continuity(slim_state* s, double dt, void* stream);

/* slim_rhs2d: for SLIM_SCHEME_TRACER, the depth-integrated horizontal residual of
 * T = 1 per 2D node (the right-hand side of Eq. 2 in weak form), 3*n_tri doubles.
 * For SLIM_SCHEME_SPLIT, the 2D external-mode residual of Eqs. 2 and 10 without
 * the 3D source (mass, then the two momentum components: 9*n_tri doubles) at
 * time t (open-boundary elevation) of the state's eta, Qx, Qy. */
slim_status slim_rhs2d(slim_state* s, double t, double* out_dev, void* stream);

/* slim_vertical_solve: one implicit vertical solve per vertex column,
 *   (M - beta_dt A) x = rhs + beta_dt b
 * M the lumped 2x2-per-layer mass at the state's elevation, A the vertical
 * upwind advection by the state's W plus SIPG diffusion (kappa_v for T/S, nu_v
 * for U/V), b the prescribed boundary fluxes (Sec. 2.4 system, 2x2 blocks per
 * layer).  With slim_params.vertical = 1: one solve per prism column of the
 * coupled system (consistent mass, 6x6 blocks, W read as the nodal Omega).
 * rhs_dev, out_dev: 6P elements of the compute type; they may alias. */
slim_status slim_vertical_solve(slim_state* s, int field, double beta_dt, const void* rhs_dev,
                                void* out_dev, void* stream);

/* slim_hpg: density anomaly rho' = rho0 (-alpha (T - T0) + beta (S - S0)) of the
 * state's T, S and the horizontal baroclinic pressure gradient r of Eq. 8 at the
 * state's elevation: per column the system D_vu r = F of Eq. 16 (printed D_vu
 * pattern with the consistent M_h), solved top-down by Algorithm 1, with
 * F = -int v g grad_h rho' dV in weak form (central density traces on lateral,
 * top and bottom faces) and the surface value g rho'(eta) grad(eta): r is the
 * horizontal gradient of the baroclinic pressure g int_z^eta rho' dz', so
 * dr/dz = -g grad_h rho' (Eq. 8's derivative taken downward).  Writes
 * SLIM_FIELD_R_X and SLIM_FIELD_R_Y.  SLIM_SCHEME_SPLIT only. */
slim_status slim_hpg(slim_state* s, void* stream);

/* slim_step: one complete internal step t -> t + dt of the state's scheme.
 * SLIM_SCHEME_TRACER: continuity, then three SSP-RK3 stages for T, then eta <-
 * eta'.  SLIM_SCHEME_SPLIT: the two-stage split-IMEX step with 2D subcycles. */
slim_status slim_step(slim_state* s, double t, double dt, void* stream);

/* slim_tracer_mass: sum over all nodes of (M T) for field T or S at the state's
 * elevation (M the lumped mass, or the consistent one with slim_params.vertical =
 * 1: the quantity each step conserves), accumulated in double with compensated
 * (Neumaier) sums in a fixed order (deterministic).  Writes one double to
 * *mass_host; synchronises. */
slim_status slim_tracer_mass(slim_state* s, int field, double* mass_host, void* stream);

/* slim_tracer_mass_noalloc: the same sum as slim_tracer_mass (the same two
 * reduction kernels, so the same bits), for callers that must not allocate device
 * memory during the call: a pool or caching allocator that forbids direct
 * cudaMalloc/cudaFree, code that must not block or synchronize the host, or a
 * fixed device-memory budget.  The paper has no counterpart; this is a library
 * convenience.
 *   mass_dev: caller-owned device address of one double, written when the
 *             stream reaches the call (nothing is copied to the host; after the
 *             first call on a device the call does not wait for the GPU).
 * Scratch: the block partials live in a fixed 1 MiB device array inside the
 * library (2 doubles per thread-block tile, at most 65536 tiles), held by every
 * GPU that loads the library until the process exits; a mesh with more tiles is
 * rejected with SLIM_ERR_ARG.  The first call on a device looks up that array's
 * device address (cudaGetSymbolAddress) with the device current, and the first
 * call per device, precision and tile size may load the kernels' module (lazy
 * loading): such a call can block the host while that happens.  Make that first
 * call before any stream capture and outside code that must not block.  The array is shared by all calls and keeps
 * the last call's partials: calls whose work overlaps on the GPU (other streams,
 * other states, other threads) race on it.  No cudaMalloc, cudaFree or
 * allocating library routine is called.  field: SLIM_FIELD_T or _S. */
slim_status slim_tracer_mass_noalloc(slim_state* s, int field, double* mass_dev, void* stream);

/* ---------------------------------------------------------------------------
 * Partitioned step on one device (Sec. 3, "Multi-GPU": horizontal domain
 * decomposition with one ghost-triangle layer, halo exchanges after every phase
 * that reads lateral neighbours, boundary kernels ahead of the interior ones).
 * Each partition is a state (SLIM_SCHEME_TRACER, equal precision and column
 * system) on a slim_mesh_create_part mesh; the states and meshes stay owned by
 * the caller and must outlive the halo.
 * ------------------------------------------------------------------------- */
typedef struct slim_halo slim_halo;
/* pair_count [n_parts * n_parts]: triangles partition i sends to partition j
 *   (row i, column j; 0 on the diagonal).
 * send_tris, recv_tris: the pairs' lists concatenated in row-major (i, j) order;
 *   entry q of pair (i, j) is an owned triangle of i (its local id) and the local
 *   id of its ghost copy in j.  Columns must have equal layer counts.
 * Allocates per pair a send and a receive buffer of one 3D field's columns, two
 * streams (the boundary stream at the highest priority) and events.
 * Errors: SLIM_ERR_ARG (null, counts, ids out of range), SLIM_ERR_MESH (layer
 * counts differ), SLIM_ERR_UNSUPPORTED (not the tracer scheme), SLIM_ERR_OOM. */
slim_status slim_halo_create(slim_state* const* parts, int n_parts, const int* pair_count,
                             const int* send_tris, const int* recv_tris, slim_halo** out);
void slim_halo_destroy(slim_halo* h);
/* Copy the owners' values of one field into every ghost column: a pack kernel per
 * pair into its send buffer, one device-to-device cudaMemcpyAsync per pair into
 * the receive buffer, an unpack kernel per pair.  field: SLIM_FIELD_T, _S, _U, _V,
 * _W (3D) or SLIM_FIELD_ETA (2D).  Enqueued on stream. */
slim_status slim_halo_exchange(slim_halo* h, int field, void* stream);
/* One tracer-scheme step t -> t + dt of every partition (the same arithmetic per
 * prism as slim_step): continuity over the owned tiles; three SSP-RK3 stages, each
 * with the boundary tiles on the high-priority stream, then the exchange of the
 * stage output on that stream while the interior tiles run on the second one;
 * then eta' -> eta, its exchange and the stretch of every column.  The ghost
 * columns' velocity and exterior profile are the caller's (uploaded or
 * exchanged once).  Ordered after the work already on `stream`, which waits for
 * the step's end; the host does not wait. */
slim_status slim_halo_step(slim_halo* h, double t, double dt, void* stream);

/* slim_selftest_conversions: diagnostic (no counterpart in the paper).  Runs the
 * library's integer-pipe binary32 <-> binary64 conversions (used by the mixed
 * form's 2D update) on n seeded bit patterns of every class (normal, subnormal,
 * zero, infinity, NaN, exact rounding ties) and counts the results that differ
 * from the GPU's own conversions (NaN compared as NaN).  Synchronises; writes the
 * two counts to host memory. */
slim_status slim_selftest_conversions(long long n, unsigned long long seed, long long* bad_d2f,
                                      long long* bad_f2d);

/* slim_selftest_barrier: diagnostic (no counterpart in the paper).  Runs `rounds`
 * rounds of the library's bounded grid barrier (the one between the stages of the
 * persistent 2D run) in a cooperative launch of n_blocks blocks (1..1024); block
 * skip_block (>= 0) leaves before the first round, so the others' wait runs out.
 * Writes the device error bits (4 = a bounded wait gave up) and the number of
 * arrivals to host memory; synchronises. */
slim_status slim_selftest_barrier(int n_blocks, int skip_block, int rounds, int* err_bits,
                                  int* arrivals);

/* slim_selftest_neighbour_wait: diagnostic (no counterpart in the paper).  Runs
 * `rounds` rounds of the bounded neighbour waits that separate the stages of the
 * persistent 2D run, on a ring of n_blocks blocks (2..1024) in one cooperative
 * launch: each block publishes its stage counter and waits for the blocks before
 * and after it.  Block skip_block (>= 0) leaves before the first round, so its
 * neighbours' waits run out, then theirs (one round later each).  Writes the device
 * error bits (4 = a bounded wait gave up) and the number of arrivals to host memory;
 * synchronises. */
slim_status slim_selftest_neighbour_wait(int n_blocks, int skip_block, int rounds, int* err_bits,
                                         int* arrivals);

/* slim_selftest_fma_peak: diagnostic (no counterpart in the paper).  Measures the
 * GPU's fused multiply-add throughput in the precision's compute type (FP64 for
 * SLIM_FP64, FP32 for SLIM_MIXED): 8 blocks of 256 threads per SM, each thread
 * running 8 independent FMA chains of `iters` steps, timed with CUDA events on the
 * legacy default stream after one warm-up launch.  Writes FLOP/s (2 per FMA) and
 * the timed launch's milliseconds to host memory; synchronises.  The roofline of
 * an arithmetic-bound kernel takes its denominator from this and from the unit
 * counts and clocks. */
slim_status slim_selftest_fma_peak(int precision, long long iters, double* flops_per_s, double* ms);

/* Number of kernels slim_step launches per call (for launch accounting). */
int slim_step_kernel_count(const slim_state* s);

/* ---------------------------------------------------------------------------
 * Phase timing: while profiling is on, slim_step records a CUDA event pair on
 * its stream around every kernel it launches, tagged with the phase below.
 * ------------------------------------------------------------------------- */
enum {
  SLIM_PHASE_CONTINUITY = 0,   /* elevation update + vertical flux (Eq. 2, Eq. 17)   */
  SLIM_PHASE_TRACER_STAGE = 1, /* fused horizontal residual + vertical solve         */
  SLIM_PHASE_HPG = 2,          /* density + baroclinic pressure gradient (Alg. 1)    */
  SLIM_PHASE_MOM_PRED = 3,     /* 3D horizontal momentum prediction + vertical sum   */
  SLIM_PHASE_EXT2D = 4,        /* 2D external-mode stages                             */
  SLIM_PHASE_MOMENTUM = 5,     /* 3D momentum update (implicit or explicit)          */
  SLIM_PHASE_TRACERS = 6,      /* 3D T, S update (implicit or explicit)              */
  SLIM_PHASE_MISC = 7,         /* small 2D kernels and copies                        */
  SLIM_PHASE_COUNT = 8
};
/* Start recording (at most max_launches kernel launches; later ones are not
   timed).  Errors: SLIM_ERR_ARG, SLIM_ERR_CUDA. */
slim_status slim_profile_begin(slim_state* s, int max_launches);
/* Synchronise the recorded events, write the summed milliseconds and the launch
   count of every phase to ms[SLIM_PHASE_COUNT] and launches[SLIM_PHASE_COUNT]
   (either may be NULL) and stop recording. */
slim_status slim_profile_end(slim_state* s, double* ms, int* launches);
const char* slim_phase_name(int phase);

#ifdef __cplusplus
}
#endif
#endif /* SLIM_H */
