/*
 * vapr.h -- C ABI of the GB300 (sm_103a) VaPr cost-and-gradient library.
 *
 * The path (arXiv 2310.07854, Sec. III-B iteration steps 2, 3 and 5, and
 * Sec. III-C's large tensors):
 *   vapr_fk              joint configurations q -> sphere centres P (and
 *                        optionally link transforms T)        [out_spheres]
 *   vapr_collision_cost  P -> per-configuration cost C, per-sphere
 *                        penetration D and dC/dP = G          [closest_pt,
 *                        out_vec, grad_out_spheres]
 *   vapr_backward        G (and q or T) -> joint gradient J
 *   vapr_pack / unpack   float32 <-> ExMy storage (Sec. IV-A, Sec. V-B)
 * P, D, G, J and T are stored in per-tensor ExMy formats (a
 * vapr_format_table), packed floor(32/bits) values per 32-bit word.
 *
 * Conventions shared by every entry point:
 *  - Memory: every array argument is a DEVICE pointer unless its comment
 *    says host.  The caller owns all buffers and the stream; the library
 *    allocates nothing on these calls.
 *  - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).
 *    Calls only enqueue work and return; they do not synchronise.
 *  - Errors: arguments are checked before anything is enqueued and a bad
 *    one returns a status without launching.  A launch failure returns
 *    VAPR_ERR_CUDA (vapr_last_cuda_error() gives the cudaError_t).  Nothing
 *    aborts, throws or traps.  Table contents on the device (link indices,
 *    pair indices) cannot be checked without a copy: kernels clamp them into
 *    range so no access leaves its buffer; vapr_robot_check() validates
 *    them once, synchronously, at set-up.
 *  - n == 0 is a no-op returning VAPR_OK; a configuration count above
 *    VAPR_MAX_CONFIGS returns VAPR_ERR_TOO_LARGE.
 *  - Packed layout: row r of a packed tensor starts at byte
 *    r * vapr_packed_row_bytes(row_len, fmt).  Value i of a row sits in
 *    32-bit little-endian word i / k, bits [b*(i%k), b*(i%k)+b) with
 *    b = 1+E+M and k = floor(32/b); unused high bits and the row's padding
 *    words are written as zero.  The row stride is a multiple of 16 bytes,
 *    and packed buffers must be 16-byte aligned.  FP32/FP16/BF16 rows are
 *    therefore plain float/half/bfloat16 arrays.
 *  - Rounding: float32 -> ExMy rounds to nearest, ties to even, with
 *    subnormals (Sec. V-B names the "_rn" conversions).  Special values
 *    follow the format's flags (VAPR_FMT_*); vapr_format_default() gives
 *    the flags of every standard format.
 */
#ifndef VAPR_H
#define VAPR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VAPR_OK = 0,
  VAPR_ERR_INVALID_ARG = 1,        /* NULL, negative or out-of-range argument */
  VAPR_ERR_UNSUPPORTED_FORMAT = 2, /* (E, M, flags) not a storage format */
  VAPR_ERR_MISALIGNED = 3,         /* pointer alignment rule broken */
  VAPR_ERR_CUDA = 4,               /* a CUDA call failed */
  VAPR_ERR_TIMEOUT = 5,            /* a device-side wait hit its limit */
  VAPR_ERR_TOO_LARGE = 6           /* a size above a documented maximum */
} vapr_status;

/* Limits of one robot / scene. */
#define VAPR_MAX_JOINTS 16
#define VAPR_MAX_SPHERES 128
#define VAPR_MAX_PAIRS 8128   /* all pairs of 128 spheres */
#define VAPR_MAX_CUBOIDS 1024
/* Configurations per call of any entry point that takes a configuration
 * count n (per problem for vapr_batched_*); larger n returns
 * VAPR_ERR_TOO_LARGE.  2^31 configurations of the smallest packed formats
 * already take over 170 GB. */
#define VAPR_MAX_CONFIGS ((int64_t)1 << 31)

/* Format flags (Sec. IV-A gives only bit counts; these classes are the
 * reading that agrees with IEEE half/bfloat16 and the OCP 8/6/4-bit types):
 *   VAPR_FMT_IEEE      all-ones exponent = Inf (mantissa 0) / NaN;
 *   VAPR_FMT_FN        no Inf, all-ones exponent and mantissa = NaN;
 *   neither            every code is finite;
 *   VAPR_FMT_SATFINITE overflow and Inf clamp to the largest finite value
 *                      (formats without Inf always clamp).
 * A NaN input becomes the format's positive all-ones NaN code, or its
 * largest positive finite value when it has no NaN. */
#define VAPR_FMT_IEEE 1u
#define VAPR_FMT_FN 2u
#define VAPR_FMT_SATFINITE 4u

typedef struct {
  uint8_t exp_bits;  /* E: 2..8 */
  uint8_t man_bits;  /* M: 1..23; 1+E+M <= 16, or E8M23 (float32) */
  uint8_t flags;     /* VAPR_FMT_* ; 8-exponent-bit formats need IEEE */
  uint8_t reserved;  /* 0 */
} vapr_format;

/* Storage format of each large tensor (Sec. III-C, Table II). */
typedef struct {
  vapr_format pos;    /* P: sphere centres [n][S*3]         (out_spheres) */
  vapr_format dist;   /* D: per-sphere penetration [n][S]                */
  vapr_format grad;   /* G: dC/dP [n][S*3]  (grad_out_spheres/closest_pt) */
  vapr_format jgrad;  /* J: joint gradient [n][J]                        */
  vapr_format xform;  /* T: link transforms [n][J*12], R row-major then t */
} vapr_format_table;

/* A serial revolute arm (Sec. II-B robot kinematics).  T_0 = I and
 * T_i = T_{i-1} * F_i * Rz(q_i); sphere s rides on link sphere_link[s],
 * c_s = T_link * [p_s; 1].  All arrays are device memory, 16-byte aligned. */
typedef struct {
  int32_t n_joints;            /* J, 1..VAPR_MAX_JOINTS */
  int32_t n_spheres;           /* S, 1..VAPR_MAX_SPHERES */
  int32_t n_pairs;             /* self-collision pairs, 0..VAPR_MAX_PAIRS */
  int32_t reserved;            /* 0 */
  const float* joint_fixed;    /* [J][12]: F_i, row-major 3x3 then translation */
  const float* sphere_local;   /* [S][4]: x, y, z in the link frame, radius */
  const int32_t* sphere_link;  /* [S]: link index 1..J */
  const int32_t* pairs;        /* [n_pairs][2]: sphere indices */
  const void* tables;          /* NULL, or tables that vapr_robot_tables_build
                                  made for this robot (see there); they change
                                  how fast a launch starts, never a result */
} vapr_robot;

/* ---- robot tables (robot preprocessing) ------------------------------------
 * Every launch that runs the collision stage (vapr_collision_cost,
 * vapr_cost_grad, vapr_cost_grad_noalloc, vapr_cost_grad_fused, the
 * multi-problem launch) first lays out, in each block's shared memory, the
 * robot's spheres grouped by link, its self-collision clusters (runs of up
 * to 3 spheres of one link), its self pairs grouped by cluster pair (the
 * self-collision broad phase of iteration step 3, Sec. III-B) and the
 * fixed-point exponent of the self terms' sums (from the most pairs that
 * name one sphere).  Building
 * that takes each block about 10 us for an arm with 832 pairs; with
 * robot->tables set, the blocks copy tables built once instead.  Each
 * launch checks on the device that the tables were built for the robot's
 * current joint, sphere, link and pair words (a hash) and are intact (a
 * checksum of the tables themselves), and otherwise builds its own, so stale
 * or damaged tables cost speed, never correctness.  The tables do
 * not depend on the cost parameters. */
/* bytes of the tables of `robot` (0 when the robot is invalid) */
size_t vapr_robot_tables_bytes(const vapr_robot* robot);
/* Builds the tables of `robot` (robot->tables is ignored) into `tables`
 * (device memory, 16-byte aligned, bytes >= vapr_robot_tables_bytes);
 * VAPR_ERR_INVALID_ARG when the buffer is missing or too small.
 * Asynchronous on `stream`; the buffer is the caller's and must outlive the
 * launches that use it. */
vapr_status vapr_robot_tables_build(const vapr_robot* robot, void* tables, size_t bytes, void* stream);

/* Oriented cuboids (device memory, 16-byte aligned). */
typedef struct {
  int32_t n_cuboids;           /* O, 0..VAPR_MAX_CUBOIDS */
  int32_t reserved;
  const float* pose;           /* [O][12]: rotation row-major, then centre */
  const float* half_ext;       /* [O][3]: half side lengths (> 0) */
  const void* grid;            /* NULL, or a broad-phase grid that
                                  vapr_scene_grid_build made for this scene
                                  (see there); it changes which cuboids the
                                  environment loop visits, never a result */
} vapr_scene;

/* ---- broad-phase grid (scene preprocessing) --------------------------------
 * A uniform grid of cubic cells over the region where a sphere of radius
 * <= reach can pass a cuboid's bounding test (centre distance below
 * r + eta + half diagonal), each cell holding the bitmask of the cuboids
 * whose test a sphere centred in it can pass.  With scene->grid set, the
 * collision stage (vapr_collision_cost, vapr_cost_grad, vapr_ik_*,
 * vapr_surrogate_collision_cost, vapr_swept_cost) visits only the cuboids
 * of a sphere's (or swept point's) cell, in cuboid order, with the same
 * bounding test and exact distance: its outputs are bit-identical to the
 * plain loop over every cuboid.  Each launch checks on the device that the
 * grid was built for the scene's current pose and half-extent words (a
 * hash), the same eta and sphere radii all in [0, reach], and otherwise
 * runs the plain loop, so a stale grid costs speed, never correctness.
 * The multi-problem launch uses each problem's scene grid the same way. */
#define VAPR_GRID_MAX_CELLS 128
/* bytes of a grid for n_cuboids cuboids and at most cells_per_axis cells
 * along each axis (1..VAPR_GRID_MAX_CELLS); 0 when out of range */
size_t vapr_scene_grid_bytes(int32_t n_cuboids, int32_t cells_per_axis);
/* Builds the grid of `scene` (scene->grid is ignored) into `grid` (device
 * memory, 16-byte aligned, grid_bytes >= vapr_scene_grid_bytes), for
 * spheres of radius <= reach and this eta.  The cell side is the region's
 * longest extent / cells_per_axis.  Asynchronous on `stream`; the grid
 * buffer is the caller's and must outlive the launches that use it.  A
 * scene whose bounding region is not finite, or wider than 1e6 m, gets a
 * grid marked unusable (the plain loop runs). */
vapr_status vapr_scene_grid_build(const vapr_scene* scene, float reach, float eta,
                                  int32_t cells_per_axis, void* grid, size_t grid_bytes,
                                  void* stream);

/* Cost parameters (reading; the paper delegates them to CuRobo):
 * D_s = sum_o max(0, r_s + eta - d_o(c_s)),
 * P_ij = max(0, r_i + r_j + eta_self - |c_i - c_j|),
 * C = w_coll * sum_s D_s + w_self * sum_pairs P_ij. */
typedef struct {
  float eta, eta_self, w_coll, w_self;
} vapr_cost_params;

/* ---- status and formats (host only, no device work) ---------------------- */
const char* vapr_status_string(vapr_status s);
/* the cudaError_t of the last VAPR_ERR_CUDA on this thread (0 if none) */
int vapr_last_cuda_error(void);
/* flags of the standard format with these bit counts (see VAPR_FMT_*) */
vapr_format vapr_format_default(int exp_bits, int man_bits);
/* 1 if f is a supported storage format, else 0 */
int vapr_format_supported(vapr_format f);
/* bytes of one packed row of row_len values (a multiple of 16; 0 when
 * row_len <= 0 or f is unsupported) */
size_t vapr_packed_row_bytes(int64_t row_len, vapr_format f);

/* Reads and clears the sticky error words of kernels with device-side waits
 * (the TMA staging wait of vapr_backward, the pipeline waits of the
 * tensor-core kernels): *code receives VAPR_ERR_TIMEOUT if a wait hit its
 * limit since the last call, else 0.  Synchronous. */
vapr_status vapr_device_error(int32_t* code);

/* Copies the robot's device tables to the host and checks them: links in
 * 1..J, pair indices in 0..S-1 and distinct, radii >= 0.  Synchronous.
 * Returns VAPR_ERR_INVALID_ARG on the first bad entry. */
vapr_status vapr_robot_check(const vapr_robot* robot);

/* ---- converters (Sec. IV-A packing, Sec. V-B "_rn" conversion) ---------- */
/* src: float32 [rows][row_len] (contiguous, 4-byte aligned);
 * dst: packed rows (16-byte aligned), row stride vapr_packed_row_bytes. */
vapr_status vapr_pack(const float* src, int64_t rows, int64_t row_len,
                      vapr_format f, void* dst, void* stream);
/* the inverse: exact decode of every code to float32 */
vapr_status vapr_unpack(const void* src, int64_t rows, int64_t row_len,
                        vapr_format f, float* dst, void* stream);

/* ---- the path ------------------------------------------------------------ */
/* Forward kinematics (Sec. II-B; iteration step 2 of Sec. III-B).
 * q: float32 [n][J] (4-byte aligned).  pos_packed: [n] rows of S*3 values
 * in table->pos.  xform_packed: NULL, or [n] rows of J*12 values (T_1..T_J,
 * each R row-major then t) in table->xform. */
vapr_status vapr_fk(const vapr_robot* robot, const float* q, int64_t n,
                    const vapr_format_table* table, void* pos_packed,
                    void* xform_packed, void* stream);

/* Collision cost (iteration steps 3-4 of Sec. III-B).
 * pos_packed: [n] rows of S*3 values in table->pos.
 * cost: NULL or float32 [n].  dist_packed: NULL or [n] rows of S values in
 * table->dist.  grad_packed: NULL or [n] rows of S*3 values of dC/dc_s in
 * table->grad.  The environment sum runs over every cuboid; the hinge's
 * gradient at exactly zero penetration is 0, and a self pair at zero
 * distance adds no gradient.  Each configuration's outputs depend on that
 * configuration alone (fixed summation orders; the self pairs' gradient
 * terms are summed as integers, u times 2^e rounded, e set by the most
 * pairs naming one sphere, so their order does not matter), whatever the
 * batch, the scene grid or the order in which the kernel's warps take
 * configurations.
 * Launches made outside stream capture may overlap one another (on other
 * streams or host threads), and so may successive replays of one
 * instantiated graph, which CUDA runs one after another.  A launch captured
 * into a graph owns one work counter for good: every executable instance
 * of that capture (a second cudaGraphInstantiate, a cudaGraphClone, the
 * graph embedded twice as a child node) shares it, so two such instances
 * must not run at the same time.  The call keeps a small host-side record
 * per device for the kernel's work counters (an event per recent launch);
 * it allocates no device memory. */
vapr_status vapr_collision_cost(const vapr_robot* robot, const vapr_scene* scene,
                                const vapr_cost_params* params,
                                const void* pos_packed, int64_t n,
                                const vapr_format_table* table, float* cost,
                                void* dist_packed, void* grad_packed,
                                void* stream);

/* Backward kinematics (iteration step 5 of Sec. III-B):
 * J_j = dC * sum_{s: link(s) >= j} G_s . (a_j x (c_s - o_j)), a_j and o_j
 * the z-axis and origin of T_j.  q: float32 [n][J].  xform_packed: NULL to
 * recompute FK from q, else the rows vapr_fk wrote (table->xform).
 * grad_packed: rows of S*3 values in table->grad.  dcost: NULL (= 1) or
 * float32 [n].  jgrad_packed: [n] rows of J values in table->jgrad.
 * Zero gradient words are skipped (Sec. III-C sparsity). */
vapr_status vapr_backward(const vapr_robot* robot, const float* q,
                          const void* xform_packed, const void* grad_packed,
                          const float* dcost, int64_t n,
                          const vapr_format_table* table, void* jgrad_packed,
                          void* stream);

/* ---- swept-sphere environment cost (trajectory optimisation) -------------- */
#define VAPR_MAX_SWEPT_SAMPLES 64

/* The environment cost of spheres swept between consecutive timesteps, whose
 * gradient is closest_pt_swept (Sec. III-C names the tensor; the paper
 * prints no formula, this is the library's reading).  The n rows of
 * pos_packed are trajectories of `horizon` consecutive configurations.  Row
 * h sweeps each sphere toward row h' = h+1 (h' = h on a trajectory's last
 * row) at K = samples points p_k = c_h + (k/K)(c_h' - c_h), k = 0..K-1:
 *   D_s = sum_k sum_o max(0, r_s + eta - d_o(p_k)),  cost = w_coll sum_s D_s,
 *   G_s = d(total swept cost of the trajectory)/dc_s of this row: the row's
 *   own points weighted 1 - k/K (1 on a last row) plus the previous row's
 *   points weighted k/K.
 * Self-collision is not part of it (vapr_collision_cost has it).  With
 * samples = 1 the results equal vapr_collision_cost's environment term
 * bit for bit.  Formats: P in table->pos, D in table->dist, G in
 * table->grad.  n % horizon == 0, 1 <= samples <= VAPR_MAX_SWEPT_SAMPLES.
 * cost (float32 [n]), dist_packed and grad_packed may each be NULL. */
vapr_status vapr_swept_cost(const vapr_robot* robot, const vapr_scene* scene,
                            const vapr_cost_params* params, const void* pos_packed, int64_t n,
                            int32_t horizon, int32_t samples, const vapr_format_table* table,
                            float* cost, void* dist_packed, void* grad_packed, void* stream);

/* ---- compute ceiling of the environment pair test (measurement) ---------- */
/* The collision stage is bound by FP32 arithmetic, not by memory, so its
 * roofline needs a compute ceiling; this call measures one.  The paper has
 * no counterpart: it is a measurement aid of this library.
 * It runs the collision stage's own environment loop (Sec. III-B step 3:
 * per sphere and cuboid, the bounding-sphere test, then the exact box term
 * where it passes, two spheres per lane, cuboids in shared memory) on
 * sphere centres held in registers, repeating it `reps` times per group of
 * 64 spheres, with no packed rows, no self pairs and no scene grid.  On
 * spheres that clear every cuboid the loop is the bounding tests alone, so
 * n * n_cuboids * reps / time is the GPU's rate of the method's pair tests.
 *  - spheres: float32 [n][4] (x, y, z, r), device, 16-byte aligned.
 *  - out: float32 [n][4], device, 16-byte aligned: per sphere the
 *    environment term of vapr_collision_cost with these margins,
 *    (D_s = sum_o max(0, r + eta - d_o(c)), G_s = w_coll dD_s/dc), from the
 *    last repetition (every repetition computes the same values).
 *  - reps >= 1; n = 0 does nothing.  scene->grid is ignored.
 *  - Errors: INVALID_ARG (NULL pointers, n < 0, reps < 1), MISALIGNED,
 *    TOO_LARGE (n_cuboids), CUDA.  Asynchronous on the stream. */
vapr_status vapr_env_ceiling(const vapr_scene* scene, const float* spheres, int64_t n,
                             float eta, float w_coll, int32_t reps, float* out, void* stream);

/* Warps one vapr_env_ceiling launch keeps resident on the current device
 * for a scene of n_cuboids (every SM full); each warp takes 64 spheres at a
 * time, so n a multiple of 64 times this count gives every warp the same
 * work.  0 on error (no device, n_cuboids out of range). */
int64_t vapr_env_ceiling_warps(int32_t n_cuboids);

/* ---- IK optimisation iteration (Sec. III-B, iteration steps 1-7) --------- */
/* A batch of IK seeds optimised on the GPU around the cost-and-gradient
 * path.  Each iteration (vapr_ik_step) evaluates every seed at N step
 * scales along its direction (FK, collision cost, backward pass, then the
 * pose and bound terms), keeps the lowest-cost scale (the paper's line
 * search over N), and computes the next L-BFGS direction.  Total cost:
 *   collision (vapr_collision_cost) + w_pos |t - t*|^2 + w_rot |R - R*|_F^2
 *   + w_bound sum_j (max(0, q_j - hi_j)^2 + max(0, lo_j - q_j)^2),
 * (R, t) the last link frame T_J.  When the best scale is 0 the history is
 * cleared and the direction restarts from steepest descent scaled so that
 * its largest joint move is step0.  Readings: the paper lists these costs
 * and steps but prints no formula. */
#define VAPR_IK_MAX_SCALES 16
#define VAPR_IK_MAX_HISTORY 16

typedef struct {
  float w_pos, w_rot, w_bound;
  float step0;                        /* largest joint move of a restart direction (rad) */
  int32_t n_scales;                   /* N, 1..VAPR_IK_MAX_SCALES */
  int32_t history;                    /* L-BFGS pairs kept, 1..VAPR_IK_MAX_HISTORY */
  float scales[VAPR_IK_MAX_SCALES];   /* step scales, scales[0..N) */
  const float* q_lo;                  /* device float32 [J] joint limits */
  const float* q_hi;
} vapr_ik_params;

/* Workspace of vapr_ik_init / vapr_ik_step for n_seeds seeds: the solver
 * state (gradient, direction, history) and the N x n_seeds candidates with
 * their path intermediates.  0 on a bad argument. */
size_t vapr_ik_workspace_bytes(const vapr_robot* robot, int64_t n_seeds, const vapr_ik_params* ik,
                               const vapr_format_table* table);

/* Starts the solver at q (device float32 [n_seeds][J]): cost and gradient
 * at q, steepest-descent direction, empty history.  goal: device float32
 * [n_seeds][12] (R* row-major, then t*).  cost: NULL or float32 [n_seeds]. */
vapr_status vapr_ik_init(const vapr_robot* robot, const vapr_scene* scene,
                         const vapr_cost_params* params, const vapr_ik_params* ik,
                         const float* goal, const float* q, int64_t n_seeds,
                         const vapr_format_table* table, void* workspace, size_t workspace_bytes,
                         float* cost, void* stream);

/* One iteration; q (device float32 [n_seeds][J]) is updated in place.
 * cost: NULL or float32 [n_seeds] (after the step); pick: NULL or int32
 * [n_seeds] (index of the kept scale).  The workspace must come from
 * vapr_ik_init with the same arguments. */
vapr_status vapr_ik_step(const vapr_robot* robot, const vapr_scene* scene,
                         const vapr_cost_params* params, const vapr_ik_params* ik,
                         const float* goal, float* q, int64_t n_seeds,
                         const vapr_format_table* table, void* workspace, size_t workspace_bytes,
                         float* cost, int32_t* pick, void* stream);

/* ---- tensor-core GEMM (building block of the learned surrogate) ----------- */
/* C = A * B^T on the tcgen05 tensor cores (TMA-fed shared memory, FP32
 * accumulation in tensor memory).  A: bfloat16 [M][K], B: bfloat16 [N][K],
 * both row-major with K contiguous; C: float32 [M][N] row-major.
 * M % 128 == 0, N % 256 == 0, K % 64 == 0 and K > 0 (INVALID_ARG otherwise);
 * A, B, C 16-byte aligned. */
vapr_status vapr_gemm_bf16(const void* A, const void* B, float* C, int64_t M, int64_t N,
                           int64_t K, void* stream);

/* ---- the whole step ------------------------------------------------------ */
/* Device workspace that vapr_cost_grad needs for n configurations: the
 * packed P and G rows, each region 256-byte aligned.  0 on a bad argument. */
size_t vapr_cost_grad_workspace_bytes(const vapr_robot* robot, int64_t n,
                                      const vapr_format_table* table);

/* One step of the path, q -> (C, D, J): vapr_fk, vapr_collision_cost and
 * vapr_backward back to back on `stream` (iteration steps 2-5 of
 * Sec. III-B), with P and G held in the caller's workspace in their table
 * formats and FK recomputed in backward.  q: float32 [n][J].  dcost: NULL
 * (= 1) or float32 [n].  cost: float32 [n] (required).  dist_packed: NULL or
 * [n] rows of S values (table->dist).  jgrad_packed: [n] rows of J values
 * (table->jgrad).  workspace: device, 256-byte aligned, at least
 * vapr_cost_grad_workspace_bytes(robot, n, table) bytes (INVALID_ARG if
 * smaller); its contents are scratch.  Results equal the three calls made
 * one by one. */
vapr_status vapr_cost_grad(const vapr_robot* robot, const vapr_scene* scene,
                           const vapr_cost_params* params, const float* q, int64_t n,
                           const vapr_format_table* table, const float* dcost, float* cost,
                           void* dist_packed, void* jgrad_packed, void* workspace,
                           size_t workspace_bytes, void* stream);

/* The same step as vapr_cost_grad in one kernel, with the sphere centres P
 * and their gradient G kept on the SM, never written to device memory: the
 * fused upper bound of the staged design (not storing the large tensors at
 * all, against storing them in reduced formats, Sec. III-C).  P and G are
 * still rounded to table->pos and table->grad in registers, as storing and
 * loading them would.  Same arguments as vapr_cost_grad without the
 * workspace.  cost, the D rows and the joint gradient equal
 * vapr_cost_grad's bit for bit (the same collision code on the same rounded
 * centres, and the backward sums taken in the same order with the same
 * operations). */
vapr_status vapr_cost_grad_fused(const vapr_robot* robot, const vapr_scene* scene,
                                 const vapr_cost_params* params, const float* q, int64_t n,
                                 const vapr_format_table* table, const float* dcost, float* cost,
                                 void* dist_packed, void* jgrad_packed, void* stream);

/* ---- many uneven problems in one persistent launch ------------------------ */
/* One planning problem of an uneven batch (device pointers, as for
 * vapr_cost_grad): its own arm tables, obstacles, parameters,
 * configurations and outputs.  Configuration counts, horizons and cuboid
 * counts may all differ between problems; the format table is shared. */
typedef struct {
  vapr_robot robot;
  vapr_scene scene;
  vapr_cost_params params;
  const float* q;        /* [n][J] */
  int64_t n;             /* configurations: trajectories x horizon */
  const float* dcost;    /* NULL (= 1) or [n] */
  float* cost;           /* [n] */
  void* dist_packed;     /* NULL or [n] rows of S values (table->dist) */
  void* jgrad_packed;    /* [n] rows of J values (table->jgrad) */
  int32_t deferred;      /* 0: ready at plan time; 1: waits for vapr_batched_publish */
  int32_t reserved;      /* 0 */
} vapr_problem;

typedef struct {
  int32_t tile;          /* configurations per work item: 32, 64, 128 or 256 */
  int32_t wait_limit_us; /* bound on the wait for a deferred problem; 0 = 1 s */
} vapr_batch_tuning;

/* Opaque host-side handle of a plan (filled by vapr_batched_plan). */
typedef struct {
  uint64_t opaque[160];
} vapr_batch_plan;

/* Device bytes of the plan of this batch: problem descriptors, the work
 * list, per-problem ready words, a work counter and one scratch slice per
 * resident block for the packed P and G rows of a tile.  0 on a bad argument. */
size_t vapr_batched_plan_bytes(const vapr_problem* problems, int32_t n_problems,
                               const vapr_format_table* table, const vapr_batch_tuning* tuning);

/* Builds the plan into plan_dev (device, 256-byte aligned, at least
 * vapr_batched_plan_bytes) and fills the host handle.  problems is a HOST
 * array.  Work items are (problem, tile of configurations) pairs, ordered
 * by estimated cost, longest first.  Synchronous (it copies the descriptors
 * to the device); call it once per batch shape, outside stream capture. */
vapr_status vapr_batched_plan(const vapr_problem* problems, int32_t n_problems,
                              const vapr_format_table* table, const vapr_batch_tuning* tuning,
                              void* plan_dev, size_t plan_bytes, vapr_batch_plan* plan);

/* Marks a deferred problem ready (a device write on `stream`). */
vapr_status vapr_batched_publish(const vapr_batch_plan* plan, int32_t problem, void* stream);

/* Evaluates every problem of the plan: one persistent launch in which each
 * block claims work items from the counter and runs FK, the collision cost
 * and the backward pass on the tile (results equal vapr_cost_grad per
 * problem).  Enqueues a reset of the counter and of *dev_status, then the
 * launch; both are stream work.  dev_status: device int32 that ends as 0, or
 * VAPR_ERR_TIMEOUT when a deferred problem was not published within the
 * wait limit (its items are then skipped and the others still run). */
vapr_status vapr_batched_eval(const vapr_batch_plan* plan, int32_t* dev_status, void* stream);

/* ---- the whole step without allocation ------------------------------------ */
/* Size of the library's fixed device scratch array (64 MiB per GPU that
 * loads the library, held until the process exits). */
#define VAPR_NOALLOC_SCRATCH_BYTES (64u << 20)

/* vapr_cost_grad for callers that cannot allocate device memory while they
 * run: a real-time planning or control loop whose latency budget cannot
 * absorb cudaMalloc (which may synchronise the device), or a program whose
 * device memory is fixed at start-up or owned by another allocator.  The
 * paper has no counterpart; it is an addition of this library.
 *  - Same arguments and results as vapr_cost_grad, minus the workspace: the
 *    P and G rows live in a fixed array inside the library.  The caller
 *    still passes (and owns) every input and output.
 *  - Nothing is allocated: no cudaMalloc, cudaFree or allocating library
 *    call.  The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current and caches it; make
 *    that first call before any stream capture.  The cached address is not
 *    looked up again, so it does not survive cudaDeviceReset (which
 *    recreates the device's context): a process that resets a device must
 *    not call this entry point on that device afterwards.
 *  - Returns VAPR_ERR_TOO_LARGE when vapr_cost_grad_workspace_bytes(robot,
 *    n, table) exceeds VAPR_NOALLOC_SCRATCH_BYTES (FP32 storage with 52
 *    spheres: up to 53,773 configurations per call).
 *  - Every call shares the one array and it keeps the last call's contents;
 *    nothing in it needs to start at zero.  Calls whose work overlaps on the
 *    GPU (other streams, other host threads) race on it: serialise them. */
vapr_status vapr_cost_grad_noalloc(const vapr_robot* robot, const vapr_scene* scene,
                                   const vapr_cost_params* params, const float* q, int64_t n,
                                   const vapr_format_table* table, const float* dcost,
                                   float* cost, void* dist_packed, void* jgrad_packed,
                                   void* stream);

/* ---- learned signed-distance surrogate ------------------------------------ */
/* A per-scene network estimating the scene signed distance
 * sdf(p) = min_o d_o(p) (the box distance of vapr_collision_cost), used as a
 * broad phase in front of the exact collision test.  The paper has no
 * counterpart; the library adds it.  The network, of domain coordinates u:
 *   f(u) = w4 . s(W3 s(W2 s(W1 u + b1) + b2) + b3) + b4,  s(z) = z/(1+e^-z)
 * with hidden width 256.  The two 256 x 256 layers run on the tcgen05 tensor
 * cores: bfloat16 weights and activations, float32 accumulation; layer 1,
 * the biases, the output dot product and the master weights are float32.
 * Parameters (float32) in this order, W rows being output units:
 *   W1[256][3], b1[256], W2[256][256], b2[256], W3[256][256], b3[256],
 *   w4[256], b4  (VAPR_MLP_PARAMS values). */
#define VAPR_MLP_HIDDEN 256
#define VAPR_MLP_PARAMS (2 * 256 * 256 + 7 * 256 + 1)

/* Bytes of a network state (device memory the caller allocates, 256-byte
 * aligned): master parameters, Adam moments and step, bfloat16 W2, W3 and
 * their transposes. */
size_t vapr_mlp_state_bytes(void);

/* Loads parameters (device float32 [VAPR_MLP_PARAMS]) into `state`, zeroes
 * the Adam moments and step and builds the bfloat16 copies. */
vapr_status vapr_mlp_init(void* state, const float* params, void* stream);

/* Copies the master parameters out (device float32 [VAPR_MLP_PARAMS]). */
vapr_status vapr_mlp_get_params(const void* state, float* params, void* stream);

/* out[i] = f(u_i) for u float32 [n][3], out float32 [n].
 * One persistent launch: 128 inputs per tile, layer 1 on the CUDA cores,
 * layers 2 and 3 on the tensor cores with the weights streamed through
 * shared memory by TMA, the activations kept on chip. */
vapr_status vapr_mlp_forward(const void* state, const float* u, int64_t n, float* out,
                             void* stream);

/* Training workspace for batches of `batch` samples: 0 unless batch is a
 * positive multiple of 128 and at most 1 << 20. */
size_t vapr_mlp_workspace_bytes(int64_t batch);

/* Squared-error loss L = mean_i w_i (f(u_i) - y_i)^2 over one batch, with
 * w_i = over_weight where f(u_i) > y_i and 1 elsewhere (over_weight = 1: the
 * mean squared error; > 1 penalises overestimates, making the network a
 * more conservative distance estimate), and dL/dparams (same order as the
 * parameters) by the backward pass: forward GEMMs with fused bias, SiLU and
 * head epilogues, backward GEMMs for dL/dA and, split over the batch, for
 * dL/dW.  u float32 [batch][3], y float32 [batch]; over_weight > 0;
 * workspace: device, 256-byte aligned, vapr_mlp_workspace_bytes(batch)
 * bytes (INVALID_ARG if smaller); grads: NULL or float32 [VAPR_MLP_PARAMS];
 * loss: NULL or float32 [1].  Deterministic: no atomics in the sums. */
vapr_status vapr_mlp_grads(const void* state, const float* u, const float* y, int64_t batch,
                           float over_weight, void* workspace, size_t workspace_bytes,
                           float* grads, float* loss, void* stream);

/* Training hyper-parameters: Adam (Kingma and Ba) step size, moment decay
 * rates and epsilon, and the loss weight of overestimates. */
typedef struct {
  float lr, beta1, beta2, eps;
  float over_weight;
} vapr_train_params;

/* vapr_mlp_grads, then one Adam step on the master parameters (bias-corrected
 * with the state's step count, which it increments) and a refresh of the
 * bfloat16 copies.  All stream work; capturable in a CUDA graph. */
vapr_status vapr_mlp_train_step(void* state, const float* u, const float* y, int64_t batch,
                                const vapr_train_params* hp, void* workspace,
                                size_t workspace_bytes, float* loss, void* stream);

/* Exact scene signed distance sdf(p) = min_o d_o(p) of points p
 * (float32 [n][3]) -> sdf float32 [n]; +FLT_MAX with no cuboids. */
vapr_status vapr_scene_sdf(const vapr_scene* scene, const float* pts, int64_t n, float* sdf,
                           void* stream);

/* Where the network applies and how it gates the exact test. */
typedef struct {
  float lo[3], hi[3]; /* domain box: u = 2 (p - lo) / (hi - lo) - 1 */
  float pad;          /* every cuboid lies inside the box shrunk by pad metres */
  float margin;       /* a sphere takes the exact test when estimate - r < margin */
} vapr_surrogate_domain;

/* Training samples: u = domain coordinates of p, y = sdf(p) (exact) clamped
 * to [y_min, y_max] (a truncated distance: only the band near the surfaces
 * decides the gate; pass -FLT_MAX, FLT_MAX for the plain distance).
 * pts float32 [n][3] -> u float32 [n][3], y float32 [n]. */
vapr_status vapr_surrogate_samples(const vapr_scene* scene, const vapr_surrogate_domain* domain,
                                   const float* pts, int64_t n, float y_min, float y_max,
                                   float* u, float* y, void* stream);

/* The collision stage with the network as a broad phase.  For each sphere
 * centre c of each configuration the estimate is f(u(c)) inside the domain
 * box and, outside it, dist(c, box) + pad, a lower bound of sdf(c).  A
 * sphere whose estimate - r >= margin skips the sphere-cuboid tests; the
 * others, and all self-collision pairs, run the exact test of
 * vapr_collision_cost.  Results (cost, D, G) equal vapr_collision_cost
 * whenever every skipped sphere is truly clear (sdf(c) >= r + eta), which
 * holds when the network's error on the skipped spheres stays below
 * margin - eta.  estimate: float32 [n][S], written (the estimates, for
 * checking against vapr_scene_sdf).  Other arguments as vapr_collision_cost. */
vapr_status vapr_surrogate_collision_cost(const vapr_robot* robot, const vapr_scene* scene,
                                          const vapr_cost_params* params, const void* mlp_state,
                                          const vapr_surrogate_domain* domain,
                                          const void* pos_packed, int64_t n,
                                          const vapr_format_table* table, float* cost,
                                          void* dist_packed, void* grad_packed, float* estimate,
                                          void* stream);

#ifdef __cplusplus
}
#endif
#endif /* VAPR_H */
