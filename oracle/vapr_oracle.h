/*
 * FP64 CPU oracle for the VaPr batched cost-and-gradient path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this library.  It shares no code,
 * header, table or helper with the CUDA library; the two meet only through
 * the seeded inputs of paper_2310_07854_gb300/synth.py.
 *
 * What it computes (paper: Sec. III-B iteration steps 2, 3 and 5; Sec. III-C
 * large tensors; Sec. IV-A data formats; Sec. V-B conversion):
 *   - forward kinematics of a serial revolute chain to sphere centres,
 *   - the oriented-box signed distance and its gradient,
 *   - the environment-collision and self-collision costs and their gradient
 *     with respect to the sphere centres,
 *   - the joint-space gradient (backward kinematics),
 *   - an emulator of every ExMy storage format (round to nearest even).
 * The paper prints none of these formulas (it relies on CuRobo); each
 * function states the reading it follows.  Everything is computed in double
 * precision from float32 inputs.
 *
 * Parity status: every function below is pinned by tests/test_oracle_*.py
 * (closed forms, finite differences, rigid-motion invariance, brute force,
 * library casts, exhaustive code-point checks).
 */
#ifndef VAPR_ORACLE_H
#define VAPR_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Special-value classes of an ExMy format (Sec. IV-A gives only bit counts;
 * these are the readings, chosen to agree with IEEE half/bfloat16 and the
 * OCP 8/6/4-bit formats):
 *   OR_IEEE: the all-ones exponent encodes Inf (mantissa 0) and NaN.
 *   OR_FN:   no Inf; all-ones exponent with all-ones mantissa is NaN.
 *   neither: every code is a finite number.
 *   OR_SAT:  overflow and Inf clamp to the largest finite magnitude
 *            (formats without Inf always clamp). */
#define OR_IEEE 1u
#define OR_FN 2u
#define OR_SAT 4u

/* ---- ExMy emulator (Sec. IV-A, Sec. V-B "_rn") ---------------------------- */
uint32_t or_exmy_encode(float x, int E, int M, unsigned flags);
double or_exmy_decode(uint32_t code, int E, int M, unsigned flags);
double or_exmy_max_finite(int E, int M, unsigned flags);
void or_exmy_encode_batch(const float* x, int64_t n, int E, int M,
                          unsigned flags, uint32_t* codes);
/* encodes the float32 values whose bit patterns are start, start+1, ... */
void or_exmy_encode_bits_range(uint32_t start, int64_t count, int E, int M,
                               unsigned flags, uint32_t* codes);
void or_exmy_decode_batch(const uint32_t* codes, int64_t n, int E, int M,
                          unsigned flags, double* out);
/* k = floor(32/bits) codes per little-endian 32-bit word, value i of a row
 * in word i/k at bit bits*(i%k); unused bits and padding words are zero. */
void or_pack_rows(const uint32_t* codes, int64_t rows, int64_t row_len,
                  int bits, uint8_t* dst, int64_t row_stride_bytes);
void or_unpack_rows(const uint8_t* src, int64_t rows, int64_t row_len,
                    int bits, int64_t row_stride_bytes, uint32_t* codes);

/* ---- kinematics (Sec. II-B, Sec. III-B step 2) ----------------------------- */
/* T_0 = I, T_i = T_{i-1} F_i Rz(q_i); c_s = T_link(s) [p_s; 1].
 * joint_fixed [nj][12]: row-major 3x3 then translation.  sphere_local [ns][4]
 * (x, y, z, r); sphere_link [ns] in 1..nj.  xform [n][nj][12] (may be NULL),
 * pos [n][ns][3]. */
void or_fk(int nj, const float* joint_fixed, int ns, const float* sphere_local,
           const int32_t* sphere_link, const float* q, int64_t n,
           double* xform, double* pos);

/* ---- oriented-box signed distance ---------------------------------------- */
/* pose [m][12] (row-major R, then centre t), half [m][3], pts [m][3]
 * -> d [m], grad [m][3] (world-frame gradient of d). */
void or_box_sdf_batch(const float* pose, const float* half, const double* pts,
                      int64_t m, double* d, double* grad);

/* ---- collision cost (Sec. III-B step 3, Sec. III-C) ----------------------- */
/* D_s = sum_o max(0, r_s + eta - d_o(c_s));
 * P_ij = max(0, r_i + r_j + eta_s - |c_i - c_j|) over the listed pairs;
 * C = w_c sum_s D_s + w_s sum_ij P_ij;  G_s = dC/dc_s.
 * kink [n][ns] (may be NULL) is set to 1 for spheres within kink_eps of a
 * point where G is discontinuous (hinge activation, inside-argmax tie). */
void or_collision(int ns, const float* sphere_local, int npairs,
                  const int32_t* pairs, int no, const float* pose,
                  const float* half, double eta, double eta_s, double w_c,
                  double w_s, const double* pos, int64_t n, double* cost,
                  double* dist, double* grad, int32_t* kink, double kink_eps);

/* ---- backward kinematics (Sec. III-B step 5) ------------------------------ */
/* J_j = dC * sum_{s: link(s) >= j} G_s . (a_j x (c_s - o_j)), with a_j the
 * z-axis and o_j the origin of T_j, both from FK recomputed in FP64.
 * dcost may be NULL (then 1). */
void or_backward(int nj, const float* joint_fixed, int ns,
                 const float* sphere_local, const int32_t* sphere_link,
                 const float* q, const double* grad, const double* dcost,
                 int64_t n, double* jgrad);

/* ---- swept-sphere environment cost (closest_pt_swept, Sec. III-C) ------- */
/* Rows are trajectories of `horizon` consecutive configurations.  The sphere
 * s of row h is swept toward row h+1: K points p_k = (1 - a_k) c_h + a_k c_h'
 * with a_k = k / K (k = 0..K-1) and h' = h+1, or h' = h on a trajectory's
 * last row.  D_s = sum_k sum_o max(0, r_s + eta - d_o(p_k)),
 * cost = w_c sum_s D_s, and grad = d(total swept cost)/dc_h: (1 - a_k) times
 * the hinge gradient at the row's own points plus a_k times it at the
 * previous row's points (and at its own points on a last row, where h' = h).
 * kink [n][ns] (may be NULL) flags spheres with a point within kink_eps of a
 * gradient discontinuity.  pos [n][ns][3]; n a multiple of horizon. */
void or_swept(int ns, const float* sphere_local, int no, const float* pose, const float* half,
              double eta, double w_c, const double* pos, int64_t n, int horizon, int samples,
              double* cost, double* dist, double* grad, int32_t* kink, double kink_eps);

/* ---- IK optimisation iteration (Sec. III-B, iteration steps 1-7) ---------- */
/* Total cost of configurations q [n][nj] against end-effector goals
 * goal [n][12] (row-major R*, then t*; the end effector is the frame T_nj):
 *   collision cost (or_collision on the FK sphere centres)
 *   + w_pos |t - t*|^2 + w_rot |R - R*|_F^2
 *   + w_bound sum_j (max(0, q_j - hi_j)^2 + max(0, lo_j - q_j)^2),
 * and its gradient with respect to q (backward pass for the collision
 * part; for the pose part dt/dq_j = a_j x (t - o_j), dR/dq_j = [a_j]x R). */
void or_ik_costs(int nj, const float* joint_fixed, int ns, const float* sphere_local,
                 const int32_t* sphere_link, int npairs, const int32_t* pairs, int no,
                 const float* pose, const float* half, double eta, double eta_s, double w_c,
                 double w_s, double w_pos, double w_rot, double w_bound, const float* q_lo,
                 const float* q_hi, const float* goal, const float* q, int64_t n, double* cost,
                 double* grad);
/* L-BFGS direction d = -H g by the two-loop recursion over the m stored
 * pairs (s_i, y_i), oldest first ([m][dim] each), with H0 = gamma I,
 * gamma = s.y / y.y of the newest pair; m = 0 gives d = -g. */
void or_lbfgs_direction(int dim, int m, const double* s, const double* y, const double* g,
                        double* d);

/* ---- scene signed distance (surrogate labels) ----------------------------- */
/* sdf(p) = min_o d_o(p) */
void or_scene_sdf(int no, const float* pose, const float* half,
                  const double* pts, int64_t m, double* out);

/* ---- signed-distance surrogate network (project addition) ---------------- */
/* f(x) = w4 . s(W3 s(W2 s(W1 x + b1) + b2) + b3) + b4 with s(z) = z/(1+e^-z)
 * (SiLU) and hidden width H.  params (float32) in the order W1[H][3], b1[H],
 * W2[H][H], b2[H], W3[H][H], b3[H], w4[H], b4[1] (2H^2 + 7H + 1 values). */
void or_mlp_forward(const float* params, int H, const float* x, int64_t n, double* out);
/* The same network with the inputs of the two H x H layers (the activations
 * s(z1) and s(z2)) rounded to float32 and then to bfloat16 (E8M7, round to
 * nearest even) before use: the rounding points of a bfloat16 tensor-core
 * evaluation.  Weights are used as given (pass them already rounded). */
void or_mlp_forward_bf16act(const float* params, int H, const float* x, int64_t n, double* out);
/* L = mean_i w_i (f(x_i) - y_i)^2 with w_i = over_weight where f(x_i) > y_i
 * and 1 elsewhere (over_weight = 1: the mean squared error), and dL/dparams
 * (same order, double); w is piecewise constant, so dL/df_i = 2 w_i r_i / n. */
double or_mlp_grads(const float* params, int H, const float* x, const float* y, int64_t n,
                    double over_weight, double* grads);

int or_num_threads(void);
/* threads of the parallel loops over configurations from now on (n >= 1) */
void or_set_num_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
