/*
 * bpm.h -- C ABI of the GB300 batched ECC-island LLG library (libbpmllg.so).
 *
 * The library integrates the Landau-Lifshitz-Gilbert equation at 0 K for a
 * batch of exchange-coupled-composite bit-patterned islands under a moving
 * write-head field (the recording simulations of Sec. II.A and II.C of
 * Kovacs et al., "Numerical optimization of writer and media for bit
 * patterned magnetic recording", J. Appl. Phys. 120, 013902 (2016)), and
 * trains/evaluates a small MLP surrogate on the outcomes.
 *
 * Conventions shared by every entry point
 *   - Return value: BPM_OK (0) or a negative BPM_ERR_* code; the message of
 *     the last failure on the calling thread is bpm_last_error().
 *   - Ownership: the caller owns every pointer it passes; the library copies
 *     what it keeps.  Handles (bpm_ctx, bpm_batch, ids) are owned by the
 *     library and released by the matching destroy call.
 *   - Device pointers (arguments documented "device") must be device memory
 *     of the context's GPU; all work is ordered on the context's stream.
 *     Entry points taking host pointers synchronise the stream before return.
 *   - Units: nm, ps, tesla (mu0*H), A/m, J/m^3, J/m.
 *   - Magnetisation arrays are component-planar per island: m[b][c][i] at
 *     float offset (b*3 + c)*ld + i, c = x,y,z, i < n_nodes <= ld.
 *   - Initial state m = +z; "switched" means the volume-averaged m_z has
 *     reached <= 0 (writing targets -z).
 *   - Nothing blocks on the GPU without a bound: device-side waits give up
 *     after a fixed number of polls and report BPM_ERR_TIMEOUT.
 */
#ifndef BPM_H
#define BPM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define BPM_OK             0
#define BPM_ERR_ARG       (-1)   /* invalid argument (null, size, id, layout) */
#define BPM_ERR_CUDA      (-2)   /* a CUDA runtime/driver call failed */
#define BPM_ERR_OOM       (-3)   /* device allocation failed */
#define BPM_ERR_TIMEOUT   (-4)   /* a bounded device-side wait gave up */
#define BPM_ERR_NONFINITE (-5)   /* a solve produced NaN/Inf */
#define BPM_ERR_UNSTABLE  (-6)   /* an iterative solve did not converge */
#define BPM_ERR_STATE     (-7)   /* call not valid in the object's state */

/* ---- effective-field terms (term_mask bits) ---- */
#define BPM_TERM_EXCHANGE   1u   /* lumped P1 exchange */
#define BPM_TERM_ANISOTROPY 2u   /* uniaxial anisotropy */
#define BPM_TERM_DEMAG      4u   /* Fredkin-Koehler demagnetising field */
#define BPM_TERM_HEAD       8u   /* moving head-field map */
#define BPM_TERM_UNIFORM   16u   /* uniform ramped field + per-island constant field */
#define BPM_TERM_ALL       31u

/* ---- demag GEMM precision ---- */
#define BPM_PREC_FP32    0  /* FP32 operands, FP32 CUDA-core GEMM (the plain form) */
#define BPM_PREC_BF16X3  1  /* BF16 hi+lo split of both operands, three tcgen05 products
                               (hi*hi + lo*hi + hi*lo), FP32 accumulate in TMEM */
#define BPM_PREC_BF16    2  /* one BF16 tcgen05 product (hi*hi), FP32 accumulate */
#define BPM_PREC_BF16X3_REF 3  /* the BF16X3 products evaluated on CUDA cores: a slow
                                  reference for validating the tensor-core kernel */

/* ---- per-island status bits ---- */
#define BPM_ISLAND_NONFINITE 1  /* the island's state became NaN/Inf */

/* ---- operators that bpm_mesh_get_operator can export ---- */
#define BPM_OP_EXCHANGE_F32  0  /* [n][n] float: S with B_ex = -S m (tesla), as used by the kernels */
#define BPM_OP_DEMAG_F64     1  /* [3n][3n] double: N with H = -N M, index c*n+i (needs BPM_MESH_KEEP_F64) */
#define BPM_OP_DEMAG_F32     2  /* [3n][3n] float: -mu0*1e6*N, the FP32 GEMM operand (tesla per MA/m) */
#define BPM_OP_VOLUMES_F64   3  /* [n] double: lumped nodal volumes V_i (nm^3) */
#define BPM_OP_NODAL_MS_F64  4  /* [n] double: nodal Ms_i (A/m) */
#define BPM_OP_NODAL_KU_F64  5  /* [n] double: nodal Ku_i (J/m^3) */

/* ---- mesh upload flags ---- */
#define BPM_MESH_KEEP_F64  1u   /* keep the FP64 demag matrix on the device (for export) */

typedef struct bpm_ctx bpm_ctx;
typedef struct bpm_batch bpm_batch;

/* Material of one mesh region (Sec. II.B, Fig. 3; Table I row A_ex,int). */
typedef struct {
    double Ms_A_per_m;   /* saturation magnetisation */
    double Ku_J_per_m3;  /* uniaxial anisotropy constant */
    double A_J_per_m;    /* exchange stiffness */
} bpm_region_mat;

/* One island of a batch (44 bytes, 4-byte aligned). */
typedef struct {
    int32_t mesh_id;     /* mesh returned by bpm_mesh_upload */
    float   Ms_scale;    /* Ms multiplier (jitter) */
    float   Ku_scale;    /* Ku multiplier (jitter) */
    float   u[3];        /* easy axis, unit vector */
    float   pos_nm[2];   /* island centre in the media frame (x down-track, y cross-track) */
    float   Hext_T[3];   /* constant field on this island (the H_ext of Sec. II.C), tesla */
} bpm_island;

/* Run parameters shared by all islands of a batch. */
typedef struct {
    double   dt_ps;       /* output interval (0.1 ps in the workloads) */
    int32_t  substeps;    /* Heun steps per output interval (step h = dt/substeps), >= 1; or 0:
                             the library takes the stable count of bpm_stable_substeps */
    int32_t  precision;   /* BPM_PREC_* */
    double   t0_ps;       /* start time */
    double   alpha;       /* Gilbert damping */
    double   rise_ps;     /* linear rise of head and uniform field, ramp = min(1, t/rise); <= 0: none */
    double   v_m_per_s;   /* head velocity along +x (signed: < 0 moves the head along -x) */
    double   x0_nm;       /* head position at t = 0 */
    int32_t  map_id;      /* head map from bpm_headmap_upload, or -1 */
    uint32_t term_mask;   /* BPM_TERM_* */
    float    uniform_T[3];/* uniform field, ramped */
    float    pad_;
} bpm_run_params;

/* Facts about an uploaded mesh. */
typedef struct {
    int32_t n_nodes;
    int32_t n_pad;               /* node stride of a component plane (n rounded up to 32) */
    int32_t n_tets, n_boundary;
    int32_t nnz;                 /* exchange CSR entries including the diagonal */
    int32_t cg_iters_neumann, cg_iters_dirichlet;
    int32_t k_pad;               /* demag GEMM width: 3 n_pad rounded up to 64 */
    double  volume_nm3;
    double  exchange_lambda_max_T;  /* largest eigenvalue of S (nominal Ms), power iteration */
    double  field_bound_T;          /* lambda_max + max anisotropy field + mu0*max Ms */
    double  cg_residual_neumann, cg_residual_dirichlet;
} bpm_mesh_info;

/* ---------------------------------------------------------------------- */
/* Context                                                                 */
/* ---------------------------------------------------------------------- */

/* Create a context on CUDA device `device`.  cuda_stream: a cudaStream_t to
 * order all work on, or NULL for a stream the library creates.  Returns
 * BPM_ERR_CUDA if the device is absent or not sm_103. */
int  bpm_create(bpm_ctx** out, int device, void* cuda_stream);
void bpm_destroy(bpm_ctx* ctx);
/* The cudaStream_t (as void*) on which the context orders its work: the one
 * passed to bpm_create, or the library's own.  A caller that hands device
 * buffers produced or consumed on another stream orders that stream against
 * this one (events, cudaStreamWaitEvent) before and after the call. */
int  bpm_context_stream(bpm_ctx* ctx, void** cuda_stream);
/* Message of the last failure on the calling thread ("" if none). */
const char* bpm_last_error(void);
/* Library version string. */
const char* bpm_version(void);

/* ---------------------------------------------------------------------- */
/* Mesh and operators (Sec. II.A hybrid FEM/BEM, Fig. 3 media)             */
/* ---------------------------------------------------------------------- */

/* Upload one P1 tetrahedral island mesh and assemble its operators on the GPU
 * in FP64: lumped volumes, nodal Ms/Ku, the exchange operator (stored FP32,
 * difference form, sliced-ELL), and the dense Fredkin-Koehler demag matrix
 * (Neumann and Dirichlet Poisson solves by batched preconditioned CG, the
 * Lindholm double-layer matrix), stored as FP32 and as a BF16 hi/lo pair.
 *   xyz_nm     [n_nodes][3] host, node positions
 *   tets       [n_tets][4]  host, node indices, any orientation
 *   tet_region [n_tets]     host, index into mats
 *   mats       [n_regions]  host
 * Errors: BPM_ERR_ARG (bad index, degenerate tet, n_nodes > 8192),
 *         BPM_ERR_UNSTABLE (CG not converged), BPM_ERR_OOM, BPM_ERR_CUDA. */
int bpm_mesh_upload(bpm_ctx* ctx, const double* xyz_nm, int32_t n_nodes,
                    const int32_t* tets, int32_t n_tets, const int32_t* tet_region,
                    const bpm_region_mat* mats, int32_t n_regions, uint32_t flags,
                    int32_t* mesh_id_out);
int bpm_mesh_info_get(bpm_ctx* ctx, int32_t mesh_id, bpm_mesh_info* out);
/* Copy one operator (BPM_OP_*) to host memory `dst` in the dense layout
 * documented at the BPM_OP_* constant. */
int bpm_mesh_get_operator(bpm_ctx* ctx, int32_t mesh_id, int32_t which, void* dst);

/* Release a mesh's device operators and buffers; its id then names no mesh.
 * Waits for the context stream.  BPM_ERR_ARG for an unknown id,
 * BPM_ERR_STATE while a live batch integrates islands of the mesh. */
int bpm_mesh_release(bpm_ctx* ctx, int32_t mesh_id);

/* Upload a head-field map mu0*H [nz][ny][nx][3] (host, float32).  Voxel
 * (ix,iy,iz) sits at origin + h*(ix,iy,iz); x is in the head frame, y and z
 * in the media frame.  Lookups are trilinear, clamped to the grid box.
 * nx, ny, nz >= 2. */
int bpm_headmap_upload(bpm_ctx* ctx, const float* B_T, int32_t nx, int32_t ny, int32_t nz,
                       float h_nm, const float origin_nm[3], int32_t* map_id_out);

/* Release a head map (its voxels, array and texture); its id then names no
 * map.  Waits for the context stream.  BPM_ERR_ARG for an unknown id,
 * BPM_ERR_STATE while a live batch uses the map. */
int bpm_headmap_release(bpm_ctx* ctx, int32_t map_id);

/* ---------------------------------------------------------------------- */
/* Head field of a saturated main pole (Sec. II.A head model, Table I)     */
/* ---------------------------------------------------------------------- */

/* Main-pole geometry and the frame of the field map.  Axes as in a head map:
 * x down-track (the trailing edge of the pole at x = 0 on the ABS), y
 * cross-track (pole centred at y = 0), z up (nm).  The pole rises from the
 * air-bearing surface z = z_abs_nm to the yoke edge z_abs_nm + yoke_edge_nm.
 * Its ABS footprint is a trapezoid: width pole_tip_width_nm at the trailing
 * edge, narrowing towards the leading edge at the taper angle (measured from
 * the trailing edge), abs_thickness_nm deep down-track (the leading width is
 * kept at least a tenth of the trailing width).  The trailing face leans
 * down-track by the trailing edge angle and the two side faces flare
 * cross-track by the side edge angle, both from the vertical; the leading face
 * is vertical.  The side faces are not planar (the taper), so every face is
 * split into two triangles, the side faces along the diagonal from their
 * trailing corner at the ABS. */
typedef struct {
    float pole_tip_width_nm;       /* Table I: 5 .. 20 nm */
    float trailing_edge_angle_deg; /* Table I: 5 .. 45 deg */
    float side_edge_angle_deg;     /* Table I: 5 .. 45 deg */
    float taper_angle_deg;         /* Table I: 75 deg */
    float abs_thickness_nm;        /* down-track depth of the ABS footprint */
    float yoke_edge_nm;            /* height of the yoke edge above the ABS (153 nm) */
    float Js_T;                    /* saturation polarisation of the pole (CoFe: 2.4 T) */
    float z_abs_nm;                /* ABS height in the map frame */
    float z_sul_nm;                /* upper surface of the soft under-layer, below the map */
    int32_t sul_image;             /* 1: mirror the pole in the under-layer; 0: no under-layer */
    float trailing_shield_gap_nm;  /* Table I: 5 .. 20 nm; 0: no trailing shield */
    float shield_thickness_nm;     /* Table I: 3 .. 20 nm, the shield's height above the ABS */
    float shield_panel_nm;         /* edge length of the shield's boundary-element panels (0: 2 nm) */
    float side_shield_gap_nm;      /* Table I: 5 .. 20 nm; 0: no side shields */
} bpm_pole_geometry;

/* Field mu0*H (tesla) of the saturated main pole on a voxel grid: the pole is
 * uniformly magnetised at Js along -z, so its field is that of the magnetic
 * surface charges Js n_z on its faces (the face at the yoke edge is the charge
 * sheet that stands in for the yoke, return pole and coil); a soft under-layer
 * of unbounded permeability is the pole's mirror image in z = z_sul_nm with
 * charges of the opposite sign.
 * With trailing_shield_gap_nm > 0 a trailing shield of unbounded permeability
 * responds to the pole: a block whose leading face is parallel to the pole's
 * trailing face at that gap (down-track, at the ABS), standing on the ABS,
 * shield_thickness_nm high, 30 nm deep down-track and 40 nm wider than the
 * pole tip on each side.  Its surface is an equipotential of the magnetic
 * potential and carries no net charge: a boundary-element solve for a uniform
 * charge on each of its triangular panels (collocation at the panel
 * centroids, the panel potentials in closed form, the under-layer image of the
 * shield included), by LU factorisation on the GPU in FP64.  With
 * side_shield_gap_nm > 0 two side shields join it as one body: blocks whose
 * inner faces are parallel to the pole's flared sides at that gap, as high as
 * the trailing shield, from 10 nm behind the leading edge to 0.5 nm short of
 * the trailing shield, out to its cross-track extent.
 * Each triangle's field is evaluated in closed form (its solid angle along the
 * normal plus a logarithm per edge) in FP64.
 *   B_T  [nz][ny][nx][3] float32: voxel (ix, iy, iz) at origin + h (ix, iy, iz);
 *        host memory, or device memory of the context when on_device is 1
 *        (written in stream order on the context stream)
 * BPM_ERR_ARG for a bad geometry (non-positive sizes or Js, angles outside
 * [0, 80) deg, a taper outside (0, 90] deg, z_sul above the ABS, a shield
 * without thickness, a side gap of 40 nm or more, panels below 0.5 nm or more
 * than 6144 of them) or a grid
 * that reaches the ABS or, with the image, the under-layer;
 * BPM_ERR_UNSTABLE if the shield solve's residual exceeds 1e-8 of its scale. */
int bpm_head_field_solve(bpm_ctx* ctx, const bpm_pole_geometry* g, int32_t nx, int32_t ny, int32_t nz,
                         float h_nm, const float origin_nm[3], float* B_T, int on_device);

/* ---------------------------------------------------------------------- */
/* Batched LLG (Sec. II.C recording simulations, one batch of islands)     */
/* ---------------------------------------------------------------------- */

/* Integrator step count (Sec. II.A names the LLG solver but not its time step;
 * the explicit Heun step is stable on the fastest precession mode when
 * gamma/(1+alpha^2) |B| h <= 1/2).  For field_bound_T the largest |B_eff|
 * (tesla) a run can see, *substeps = the smallest k >= 1 with
 *   gamma/(1+alpha^2) * field_bound_T * dt_ps / k <= 1/2,
 * gamma = 0.176085963023 rad/(ps T).  Host arithmetic only (no GPU needed).
 * BPM_ERR_ARG for a negative bound, dt <= 0, alpha < 0 or a NULL output. */
int bpm_substeps_for_bound(double field_bound_T, double dt_ps, double alpha, int32_t* substeps);
/* The step count and field bound of a run of the islands isl [B] (host) under
 * p (p->substeps is ignored).  The bound is the largest over the meshes of
 * the batch of
 *   lambda_max(S) / min Ms_scale          exchange (largest eigenvalue of the
 *                                         mesh's exchange operator, power iteration)
 * + max_i (2 Ku_i / Ms_i) * max (Ku_scale / Ms_scale)      anisotropy
 * + mu0 max_i Ms_i * max Ms_scale                          demag
 * + max |B| over the head map's voxels (when p->map_id >= 0)
 * + |p->uniform_T| + max |Hext_T|                          applied fields
 * with the jitter extremes taken over the islands of that mesh.  A run with
 * p->substeps = 0 uses this k.  *field_bound_T is nullable.
 * BPM_ERR_ARG for an unknown mesh or map id or bad jitter. */
int bpm_stable_substeps(bpm_ctx* ctx, const bpm_island* isl, int32_t B, const bpm_run_params* p,
                        int32_t* substeps, double* field_bound_T);

/* Create a batch of B islands.  Islands may use different meshes (design
 * variants of uneven size): they are grouped by mesh, each group with its own
 * demag GEMM, and the groups of one output interval are captured into a
 * single CUDA graph forked over up to four streams.  Device state is
 * allocated here; the state starts at m = +z, t = p->t0_ps.  Per step of size
 * h = dt/substeps every group runs the Heun predictor and corrector (|m|
 * renormalised after each), each preceded by one demag GEMM over the group,
 * and updates the switch detector.  Magnetisation arrays passed to the batch
 * calls use a leading dimension ld >= the largest mesh's n_nodes; entries past
 * an island's own n_nodes are not read and are left untouched (reads of host
 * arrays leave them zero).
 * Errors: BPM_ERR_ARG (B < 1, unknown mesh or map id, substeps < 0). */
int bpm_batch_create(bpm_ctx* ctx, const bpm_island* isl, int32_t B,
                     const bpm_run_params* p, bpm_batch** out);
/* Set the state: m (layout above, leading dimension ld) or NULL for +z, the
 * time t0_ps, and reset the switch detector.  on_device: m is a device
 * pointer. */
int bpm_batch_set_state(bpm_batch* bt, const float* m, int32_t ld, double t0_ps, int on_device);
/* Advance by n_intervals output intervals (stream-ordered; the first call
 * captures one interval as a CUDA graph, later calls replay it). */
int bpm_batch_advance(bpm_batch* bt, int32_t n_intervals);
/* Read the state.  Any output may be NULL.
 *   m        [B][3][ld] float      switched [B] uint8 (<m_z> <= 0 now)
 *   t_sw_ps  [B] float, first crossing time, -1 if none
 *   status   [B] int32 BPM_ISLAND_* bits        mz [B] float, <m_z> now
 * on_device: all outputs are device pointers (no synchronisation). */
int bpm_batch_read(bpm_batch* bt, float* m, int32_t ld, uint8_t* switched, float* t_sw_ps,
                   int32_t* status, float* mz, int on_device);
/* Energy and torque check of the current state (the FP64 check of a run's
 * state; the paper's solver runs at 0 K, so with damping the energy of a static
 * field problem only decreases, Sec. II.A).  For every island, at the batch's
 * current time and with its run's term mask:
 *   E_J[b]          = -sum_i V_i Ms_i (B_quad,i / 2 + B_lin,i) . m_i   (J), with B_quad the
 *                     exchange, anisotropy and demag fields and B_lin the head and uniform
 *                     fields; accumulated in FP64
 *   max_torque_T[b] = max_i |m_i x B_i| (T), nullable
 * Host arrays [B] in the batch's island order.  Runs one demag product over
 * the batch (the batch's Hd buffer is recomputed by the next advance) and
 * synchronises the context stream.  BPM_ERR_TIMEOUT if a tensor-core GEMM
 * wait timed out. */
int bpm_batch_energy(bpm_batch* bt, double* E_J, float* max_torque_T);
/* Effective field B (tesla) of the current state at time t_ps, restricted to
 * term_mask, into B_out [B][3][ld] (host or device per on_device). */
int bpm_batch_field(bpm_batch* bt, double t_ps, uint32_t term_mask, float* B_out, int32_t ld,
                    int on_device);
/* Time the kernels of one integrator step with CUDA events on the context
 * stream: runs `reps` Heun steps launch by launch (outside the graph) and
 * returns the average duration in ms of one demag GEMM, one predictor stage
 * and one corrector stage.  The state advances by those steps but the batch
 * clock does not; call bpm_batch_set_state afterwards to restart a run. */
int bpm_batch_kernel_times(bpm_batch* bt, int32_t reps, double* gemm_ms, double* stage1_ms,
                           double* stage2_ms);
/* Order in which the persistent tensor-core GEMM walks a group's output tiles.
 * M-major: consecutive tiles share rows of the batch operand (the demag
 * operator is swept once per wave of CTAs); N-major: consecutive tiles share
 * rows of the operator (the batch operand is swept once per wave).  AUTO takes
 * N-major for a group whose operator has more rows than the batch, so that the
 * larger operand is read from HBM once and the smaller one is re-read from L2;
 * M-major otherwise. */
enum { BPM_RASTER_AUTO = 0, BPM_RASTER_M = 1, BPM_RASTER_N = 2 };

/* Launch configuration of a batch's kernels.  A new batch starts with
 * gemm_tile_n 256, stage_threads 256, gemm_raster AUTO, stage_islands 2,
 * gemm_k_block 32, gemm_pair 0, and streams 2 for a one-mesh batch, 1 for a
 * multi-mesh batch (the fastest on the census and uneven batches measured). */
typedef struct {
    int32_t gemm_tile_n;     /* output columns per demag-GEMM CTA: 256 or 128 */
    int32_t stage_threads;   /* threads per Heun-stage CTA: 128, 256 or 512 */
    int32_t gemm_raster;     /* BPM_RASTER_*: tile order of the tensor-core GEMM */
    int32_t stage_islands;   /* islands per Heun-stage CTA: 1 (0 = 1), or 2 with 256 threads */
    int32_t gemm_k_block;    /* K depth of a tensor-core GEMM pipeline stage: 32 (0 = 32) or 64 */
    int32_t gemm_pair;       /* 1: 256 x 256 GEMM tiles on the two SMs of a CTA pair (tcgen05
                                cta_group::2; needs gemm_tile_n 256), 0: 128 x gemm_tile_n tiles
                                on one SM */
    int32_t streams;         /* 2 .. 4: the interval graph integrates the batch as up to that many
                                chains, each on its own stream, so that one chain's GEMM overlaps
                                another chain's stage kernels: a one-mesh batch cut into chunks of
                                islands (a multiple of 128 each, the last takes the rest), a
                                multi-mesh batch's groups dealt to chains of about equal GEMM work.
                                1 (0 = 1): one chain.  Applies at the tensor-core precisions and
                                acts as 1 otherwise.  The states are bitwise the same either way. */
    double  gemm_ms;         /* measured time of one demag GEMM over the batch (autotune output) */
    double  stage_ms;        /* measured time of one predictor + one corrector over the batch */
} bpm_tuning;

/* Autotuner: time every (gemm_tile_n, gemm_raster, gemm_k_block, gemm_pair) candidate of the demag GEMM
 * and every (stage_threads, stage_islands) candidate on this batch with CUDA events (reps Heun
 * steps each, kernel by kernel), apply the fastest of each, then time reps whole intervals with
 * streams 1 .. 4 where several chains apply, and report the choice in *chosen (nullable).  The
 * state advances by the timed steps but the batch clock does not; call
 * bpm_batch_set_state afterwards to restart a run.  Tile shapes are an
 * implementation choice of this library, not of the paper. */
int bpm_batch_autotune(bpm_batch* bt, int32_t reps, bpm_tuning* chosen);
/* Apply a tuning (for example one cached from an earlier autotune). */
int bpm_batch_set_tuning(bpm_batch* bt, const bpm_tuning* t);
/* Testing aid for the failure path: raise the batch's device error flag as a
 * timed-out wait inside the tensor-core GEMM would (code != 0).  Later GEMM
 * launches of the batch then return at once, and bpm_batch_read reports
 * BPM_ERR_TIMEOUT.  code = 0 clears the flag. */
int bpm_debug_set_gemm_error(bpm_batch* bt, int32_t code);
/* Testing aid for the failure path: the time limit (ns) of the tensor-core
 * demag GEMM's waits for normal progress (copies landed, stages freed,
 * accumulators full or read back); 0 restores the default of 200 ms.  A limit
 * shorter than one output tile's MMAs (tens of microseconds) makes a real wait
 * run out: the kernel raises the batch's error flag, lets its own copies and
 * MMAs land (those waits keep the default limit), frees TMEM and returns, and
 * bpm_batch_read reports BPM_ERR_TIMEOUT.  Clear the flag with
 * bpm_debug_set_gemm_error(bt, 0) after restoring the limit. */
int bpm_debug_set_gemm_wait(bpm_batch* bt, double wait_ns);
/* Number of kernel launches in the batch's one-interval CUDA graph (the
 * graph exists after the first bpm_batch_advance; BPM_ERR_STATE before). */
int bpm_batch_graph_kernels(bpm_batch* bt, int32_t* n_kernels);
/* Current simulated time of the batch. */
int bpm_batch_time(bpm_batch* bt, double* t_ps);
int bpm_batch_destroy(bpm_batch* bt);

/* One-call form: create, advance from t0 to t0 + n_intervals*dt, read into
 * host arrays, destroy. */
int bpm_run_batch(bpm_ctx* ctx, const bpm_island* isl, int32_t B, const bpm_run_params* p,
                  int32_t n_intervals, float* m_final, int32_t ld, uint8_t* switched,
                  float* t_sw_ps, int32_t* status);
/* The same run with the outputs in caller-owned DEVICE buffers of the context's
 * device (layouts as in bpm_batch_read; any output may be NULL); the island
 * table isl stays a host array.  The copies are ordered on the context stream,
 * and the call returns after that stream has drained (the batch's scratch is
 * freed), so the outputs are ready when it returns.  Errors as bpm_run_batch,
 * including BPM_ERR_TIMEOUT for a timed-out GEMM wait. */
int bpm_run_batch_dev(bpm_ctx* ctx, const bpm_island* isl, int32_t B, const bpm_run_params* p,
                      int32_t n_intervals, float* m_final, int32_t ld, uint8_t* switched,
                      float* t_sw_ps, int32_t* status);

/* The plain form: every island integrated on its own, one island per launch,
 * with an FP32 matrix-vector demag product streaming the operator from HBM in
 * every Heun stage and single-island stage kernels (the per-island
 * recording-simulation jobs of Sec. II.C ported to the GPU as is).  Same
 * arithmetic per island as a BPM_PREC_FP32 batch; it exists as the baseline
 * that the batched path is measured against.  Outputs are host arrays as in
 * bpm_run_batch; device_ms (nullable) receives the summed CUDA-event time of
 * the integration loops. */
int bpm_run_plain(bpm_ctx* ctx, const bpm_island* isl, int32_t B, const bpm_run_params* p,
                  int32_t n_intervals, float* m_final, int32_t ld, uint8_t* switched, float* t_sw_ps,
                  int32_t* status, double* device_ms);
/* The plain form in FP64: one island per launch, every step of the recording
 * simulation (Sec. II.A, II.C) in FP64 -- the effective field from the FP64
 * exchange operator (difference form of the assembly's values), anisotropy,
 * an FP64 matrix-vector demag product with the assembly's FP64 Fredkin-Koehler
 * matrix, a trilinear head-map lookup in FP64 and the ramped uniform and
 * per-island fields; Heun predictor and corrector with |m| renormalised after
 * each; the volume-averaged m_z switch detector summed in FP64.  It is the
 * GPU twin of an FP64 reference, one island at a time, and the FP64 baseline
 * the batched path is measured against.  Every mesh used must have been
 * uploaded with BPM_MESH_KEEP_F64 (BPM_ERR_STATE otherwise); p->precision is
 * ignored.
 *   m_final  host double [B][3][ld] (nullable)   t_sw_ps host double [B], -1 if none
 *   switched, status, device_ms as in bpm_run_plain. */
int bpm_run_plain_f64(bpm_ctx* ctx, const bpm_island* isl, int32_t B, const bpm_run_params* p,
                      int32_t n_intervals, double* m_final, int32_t ld, uint8_t* switched, double* t_sw_ps,
                      int32_t* status, double* device_ms);

/* ---------------------------------------------------------------------- */
/* Surrogate MLP (stands in for the Gaussian-process predictor of the      */
/* efficient global optimisation, Sec. II.A)                               */
/* ---------------------------------------------------------------------- */

/* x[n_in] -> (Linear -> GELU) x depth (width wide) -> Linear -> n_out logits. */
typedef struct {
    int32_t n_in, width, depth, n_out;   /* e.g. 16, 256, 4, 2 */
} bpm_mlp_cfg;

/* AdamW with decoupled weight decay on the weight matrices only. */
typedef struct {
    int32_t epochs, batch;
    float   lr, weight_decay, beta1, beta2, eps;
    int32_t pad_;
} bpm_train_cfg;

/* Flat parameter layout shared by create / get / grad: for each layer l in
 * order, W_l [out][in] row-major, then b_l [out]. */

/* Create a surrogate with the given initial parameters (host, float32 [P]).
 * Training and inference run every contraction on the tensor cores with BF16
 * weights/activations and FP32 accumulation; FP32 master weights and the Adam
 * moments stay on the device. */
int bpm_surrogate_create(bpm_ctx* ctx, const bpm_mlp_cfg* cfg, const float* params, int32_t* sid);
int bpm_surrogate_param_count(bpm_ctx* ctx, int32_t sid, int64_t* count);
int bpm_surrogate_get_params(bpm_ctx* ctx, int32_t sid, float* out);
/* Mean sigmoid-BCE loss and its gradient (flat layout) on one batch X [N][n_in],
 * Y [N][n_out] (host); no parameter update. */
int bpm_surrogate_grad(bpm_ctx* ctx, int32_t sid, const float* X, const float* Y, int32_t N, float* grad,
                       float* loss);
/* Train: `epochs` passes over X, Y (host) in the given sample order, minibatches
 * of cfg->batch (the last one partial), one AdamW step per minibatch.
 * loss_curve: host [epochs * ceil(N/batch)] or NULL. */
int bpm_surrogate_train(bpm_ctx* ctx, int32_t sid, const float* X, const float* Y, int64_t N,
                        const bpm_train_cfg* cfg, float* loss_curve);
/* Probabilities sigmoid(logits) P [N][n_out] for X [N][n_in] (both host, or both
 * device if on_device, stream-ordered). */
int bpm_surrogate_infer(bpm_ctx* ctx, int32_t sid, const float* X, int64_t N, float* P, int on_device);
/* Screened error rates of designs over their jitter samples (Sec. II.C: a write
 * error is a target island that fails to switch, an adjacent-track error a
 * neighbouring island that flips).  X [n_designs * n_jitter][n_in] is
 * design-major: rows d*n_jitter .. d*n_jitter + n_jitter - 1 are the jitter
 * samples of design d.  rates [n_designs][n_out] (float64): column 0 the mean
 * over the samples of the probability that output 0's event (the target
 * switching) does NOT happen, sigmoid(-z_0); columns k >= 1 the mean
 * probability of their event, sigmoid(z_k).  Each probability is formed from
 * the logit with full relative precision on both tails and summed in FP64 in
 * a fixed order, so a run is reproducible.  X and rates are both host, or both
 * device if on_device (stream-ordered).  BPM_ERR_ARG for a bad handle, a NULL
 * pointer or a count below 1. */
int bpm_surrogate_screen(bpm_ctx* ctx, int32_t sid, const float* X, int64_t n_designs, int32_t n_jitter,
                         double* rates, int on_device);
/* Checkpoint of weights, Adam moments and step count; load needs the same shape. */
int bpm_surrogate_save(bpm_ctx* ctx, int32_t sid, const char* path);
int bpm_surrogate_load(bpm_ctx* ctx, int32_t sid, const char* path);
int bpm_surrogate_destroy(bpm_ctx* ctx, int32_t sid);

/* Size of the fixed device scratch array used by bpm_llg_advance_noalloc. */
#define BPM_NOALLOC_SCRATCH_BYTES (8 * 1024 * 1024)

/* Allocation-free advance.  The paper has no counterpart to this entry point;
 * it exists for callers that cannot allocate device memory when they step
 * islands -- for example a host application whose own pool allocator has
 * reserved the device memory, or a time-critical loop that must not stall on
 * cudaMalloc/cudaFree (which can synchronise the device).  It performs the
 * same FP32 batch advance as a BPM_PREC_FP32 batch (same kernels, same
 * arithmetic) but allocates nothing: its scratch (island table, Heun stages,
 * demag operand and field, switch-detector state, step counter) lives in one
 * fixed device array of BPM_NOALLOC_SCRATCH_BYTES bytes that every GPU which
 * loads the library holds until the process exits.
 *   isl, B      host island table, one mesh for all islands
 *   p           run parameters; p->precision must be BPM_PREC_FP32; the run
 *               starts at p->t0_ps with the switch detector reset
 *   m           device [B][3][ld]: the state at p->t0_ps on entry, the state
 *               after n_intervals intervals on return (stream-ordered)
 *   mz          device [B] volume-averaged m_z at the end, or NULL
 * Requests whose scratch would exceed the array (about 48*B*n_pad bytes, e.g.
 * 111 islands of a 1547-node mesh) fail with BPM_ERR_ARG and a message giving
 * the size needed.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress).  All calls share the one array, which keeps
 * the previous call's contents (each call clears the region it uses): calls
 * that overlap on the GPU -- on different streams or contexts of the same
 * device -- race and corrupt each other.  Work is ordered on the context's stream; the call does
 * not synchronise. */
int bpm_llg_advance_noalloc(bpm_ctx* ctx, const bpm_island* isl, int32_t B,
                            const bpm_run_params* p, int32_t n_intervals, float* m, int32_t ld,
                            float* mz);

/* ---------------------------------------------------------------------- */
/* Energy barrier in the fringing field (Sec. II.C, adjacent-track erasure) */
/* ---------------------------------------------------------------------- */

/* The paper places the adjacent bit in the head's fringing field (frozen at
 * the down-track position of the lowest barrier), computes its switching
 * barrier E_B with the nudged elastic band method, and turns it into
 * BER_adj = t_write f0 exp(-E_B / kT) (Eq. 3).  A band of n_images states of one
 * island runs from the +z minimum to the -z minimum; every image is a row of
 * one batch, so the demag products of all images of all bands are one GEMM.
 *
 * Energy (J): E = -sum_i V_i Ms_i (B_quad,i / 2 + B_lin,i) . m_i, with B_quad
 * the exchange, anisotropy and demag fields and B_lin the head and uniform
 * fields (the same terms and readings as the time integration).  Band
 * update of every image at once, in the metric <a,b> = sum_i w_i a_i . b_i
 * (w_i = V_i / sum V):
 *   force density g_i = Ms_i B_i_perp (MA/m x T), B_perp the part of the field
 *                 normal to m_i;
 *   interior image: g - <g,t> t + spring (|m+ - m| - |m - m-|) t with the
 *                 improved tangent t (the higher neighbour's side, weighted by
 *                 the energy differences at an extremum), projected on every
 *                 node's tangent plane and normalised; the highest interior
 *                 image takes g - 2 <g,t> t once climbing is on;
 *   end images:   g (they relax into the minima);
 *   m_i <- (m_i + step f_i) / |m_i + step f_i|.
 */
typedef struct {
    int32_t  n_images;     /* images per band, end images included (>= 3) */
    int32_t  max_iters;    /* band updates */
    int32_t  climb_after;  /* first update with a climbing image; < 0: never */
    int32_t  precision;    /* BPM_PREC_* of the demag product */
    int32_t  map_id;       /* head map of the fringing field, or -1 */
    uint32_t term_mask;    /* BPM_TERM_* */
    int32_t  check_every;  /* updates between convergence checks (0: 50) */
    int32_t  pad_;
    double   step;         /* > 0, per unit of force density (m^3/MJ) */
    double   spring;       /* >= 0, MA/m x T per unit of weighted distance */
    double   force_tol;    /* stop once every image's max |force_i| is below it (0: run max_iters) */
    double   head_x_nm;    /* head position: the map is sampled at x_i + pos_x - head_x, ramp 1 */
    double   uniform_T[3]; /* uniform applied field (T), added with every island's Hext_T */
} bpm_neb_params;

/* Relax one band per island.
 *   isl, D     host island table [D]; all on one mesh; each band uses its
 *              island's Ms/Ku jitter, axis, position and Hext_T
 *   m_init     host [D][n_images][3][ld] initial band, or NULL for the great
 *              circle from +z to -z through +x (uniform states)
 *   E_path     host [D][n_images] energies of the final band (J), nullable
 *   E_barrier  host [D] max over interior images of E - E of image 0 (J), nullable
 *   m_path     host [D][n_images][3][ld] final band, nullable
 *   iters_done updates run (fewer than max_iters when force_tol was met)
 *   max_force  max |force_i| over all images at the last check (MA/m x T)
 * Device buffers are allocated for the call and freed before it returns; the
 * call synchronises the context stream.  BPM_ERR_ARG on bad arguments,
 * BPM_ERR_TIMEOUT if a tensor-core GEMM wait timed out. */
int bpm_neb_run(bpm_ctx* ctx, const bpm_island* isl, int32_t D, const bpm_neb_params* p, const float* m_init,
                int32_t ld, double* E_path, double* E_barrier, float* m_path, int32_t* iters_done,
                double* max_force);

/* ---------------------------------------------------------------------- */
/* Efficient global optimisation (Sec. II.A; Jones et al. 1998)            */
/* ---------------------------------------------------------------------- */

/* The paper's optimiser fills the design space with an optimised Latin
 * hypercube (at least ten designs per parameter), describes the evaluated
 * designs with a Gaussian process, and evaluates the design of highest
 * expected improvement next, refitting after every evaluation.  Kriging model
 * on the unit cube (FP64 throughout):
 *   R_ij = exp(-sum_k theta_k (x_ik - x_jk)^2) + nugget [i == j]
 *   mu = 1'R^-1 y / 1'R^-1 1,  sigma2 = (y - mu 1)'R^-1(y - mu 1) / n
 *   nll(theta) = n ln sigma2 + ln det R   (concentrated negative log-likelihood)
 *   yhat(x) = mu + r'R^-1(y - mu 1),
 *   s2(x) = sigma2 [1 - r'R^-1 r + (1 - 1'R^-1 r)^2 / 1'R^-1 1],  r_i = R(x, x_i)
 *   EI(x) = (f_min - yhat) Phi(z) + s phi(z),  z = (f_min - yhat) / s  (f_min - yhat clipped at 0 when s = 0)
 * Limits: 2 <= n <= 2048 training designs, 1 <= d <= 64 parameters. */

/* Maximin choice among T candidate designs cands [T][n][d] (host): *best = the
 * index whose smallest squared pairwise distance is largest; min_d2 [T]
 * (nullable) receives every candidate's smallest squared distance. */
int bpm_lhs_maximin(bpm_ctx* ctx, const double* cands, int32_t T, int32_t n, int32_t d, int32_t* best,
                    double* min_d2);

/* nll for T correlation vectors theta [T][d] (host; theta_k > 0) on the data
 * X [n][d], y [n] (host); nll [T] receives +inf where R is not positive
 * definite.  One CTA factors one matrix; all T in one launch. */
int bpm_gp_nll(bpm_ctx* ctx, const double* X, const double* y, int32_t n, int32_t d, const double* theta,
               int32_t T, double nugget, double* nll);

/* Fit the kriging model at theta [d]: factor, inverse factor and weights stay
 * on the device under *gp_id; mu_sigma2 [2] (nullable) receives mu and sigma2.
 * BPM_ERR_NONFINITE if R is not positive definite. */
int bpm_gp_create(bpm_ctx* ctx, const double* X, const double* y, int32_t n, int32_t d, const double* theta,
                  double nugget, int32_t* gp_id, double* mu_sigma2);

/* yhat, s and EI below f_min at N candidates C [N][d] (host); each output
 * [N] host and nullable.  Processed in chunks of 32768 candidates. */
int bpm_gp_predict(bpm_ctx* ctx, int32_t gp_id, const double* C, int64_t N, double f_min, double* yhat,
                   double* s, double* ei);
int bpm_gp_destroy(bpm_ctx* ctx, int32_t gp_id);

#ifdef __cplusplus
}
#endif
#endif /* BPM_H */
