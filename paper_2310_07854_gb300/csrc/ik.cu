// IK optimisation iteration around the cost-and-gradient path (Sec. III-B,
// iteration steps 1-7): N step scales per seed, the path (FK, collision,
// backward) on all N x n candidates, pose and bound terms, selection of the
// lowest-cost scale, L-BFGS direction.  Kernels:
//   ik_candidates  thread per (seed, scale): q + a_k d
//   (path)         fk_kernel, collision_kernel, backward_kernel on the candidates
//   ik_terms       thread per candidate: decodes the path's joint gradient,
//                  recomputes the chain for the end-effector pose and the
//                  joint axes, adds the pose and bound terms
//   ik_update      thread per seed: argmin over the scales (lowest index on
//                  ties), history update (s.y > 0), two-loop recursion.
// Float32 throughout; deterministic.
#include "stages.cuh"

namespace vapr {

struct IkWork {
  float* g;      // [n][J] gradient at q
  float* d;      // [n][J] direction
  float* S;      // [n][m][J] a ring: pair k (0 = oldest) in slot (mhead + k) mod m
  float* Y;      // [n][m][J]
  int* mcount;   // [n]
  int* mhead;    // [n]
  float* cq;     // [n N][J] candidates
  float* ccoll;  // [n N] collision cost of the candidates
  uint8_t* cjg;  // [n N] packed joint-gradient rows (table->jgrad)
  float* ctot;   // [n N] total cost
  float* cgrad;  // [n N][J] total gradient
  uint8_t* path; // P and G rows of the candidates
  size_t P_bytes, bytes;
};

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

static IkWork carve_ik(void* base, const RobotArgs& r, int64_t n, int N, int m, const vapr_format_table* t) {
  IkWork w;
  uint8_t* b = static_cast<uint8_t*>(base);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    uint8_t* p = b ? b + off : nullptr;
    off += al256(bytes);
    return p;
  };
  const int64_t c = n * N;
  w.g = reinterpret_cast<float*>(take((size_t)n * r.J * 4));
  w.d = reinterpret_cast<float*>(take((size_t)n * r.J * 4));
  w.S = reinterpret_cast<float*>(take((size_t)n * m * r.J * 4));
  w.Y = reinterpret_cast<float*>(take((size_t)n * m * r.J * 4));
  w.mcount = reinterpret_cast<int*>(take((size_t)n * 4));
  w.mhead = reinterpret_cast<int*>(take((size_t)n * 4));
  w.cq = reinterpret_cast<float*>(take((size_t)c * r.J * 4));
  w.ccoll = reinterpret_cast<float*>(take((size_t)c * 4));
  w.cjg = take((size_t)c * row_bytes(r.J, t->jgrad));
  w.ctot = reinterpret_cast<float*>(take((size_t)c * 4));
  w.cgrad = reinterpret_cast<float*>(take((size_t)c * r.J * 4));
  w.P_bytes = (size_t)c * row_bytes(3 * (int64_t)r.S, t->pos);
  w.path = take(w.P_bytes);
  take((size_t)c * row_bytes(3 * (int64_t)r.S, t->grad));
  w.bytes = off;
  return w;
}

struct IkArgs {
  int J, N, m;
  int64_t n;
  float w_pos, w_rot, w_bound, step0;
  float scales[VAPR_IK_MAX_SCALES];
  const float* q_lo;
  const float* q_hi;
  const float* joint_fixed;  // [J][12]
  const float* goal;         // [n][12]
};

__global__ void ik_candidates(IkArgs a, const float* __restrict__ q, IkWork w, int N) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;  // candidate
  if (i >= a.n * N) return;
  const int64_t seed = i / N;
  const float al = a.scales[i - seed * N];
  for (int j = 0; j < a.J; ++j)
    w.cq[i * a.J + j] = fmaf(al, w.d[seed * a.J + j], q[seed * a.J + j]);
}

// One step of the chain: T <- T F_j Rz(q_j) (R row-major, t).
__device__ __forceinline__ void chain_step(const float* F, float qj, float R[3][3], float t[3]) {
  float B[3][3], tb[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    B[k][0] = fmaf(R[k][0], F[0], fmaf(R[k][1], F[3], R[k][2] * F[6]));
    B[k][1] = fmaf(R[k][0], F[1], fmaf(R[k][1], F[4], R[k][2] * F[7]));
    B[k][2] = fmaf(R[k][0], F[2], fmaf(R[k][1], F[5], R[k][2] * F[8]));
    tb[k] = fmaf(R[k][0], F[9], fmaf(R[k][1], F[10], fmaf(R[k][2], F[11], t[k])));
  }
  float sn, cs;
  sincosf(qj, &sn, &cs);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    R[k][0] = fmaf(cs, B[k][0], sn * B[k][1]);
    R[k][1] = fmaf(cs, B[k][1], -sn * B[k][0]);
    R[k][2] = B[k][2];
    t[k] = tb[k];
  }
}

__global__ void ik_terms(IkArgs a, IkWork w, DevFmt fj, int64_t jstride, int N) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= a.n * N) return;
  const int J = a.J;
  const float* qc = w.cq + c * J;
  const float* gl = a.goal + (c / N) * 12;
  // end-effector pose T_J
  float R[3][3] = {{1.f, 0.f, 0.f}, {0.f, 1.f, 0.f}, {0.f, 0.f, 1.f}}, t[3] = {0.f, 0.f, 0.f};
  for (int j = 0; j < J; ++j) chain_step(a.joint_fixed + 12 * j, qc[j], R, t);
  float dt[3], dR[3][3], tot = w.ccoll[c];
  for (int i = 0; i < 3; ++i) {
    dt[i] = t[i] - gl[9 + i];
    tot = fmaf(a.w_pos * dt[i], dt[i], tot);
    for (int k = 0; k < 3; ++k) {
      dR[i][k] = R[i][k] - gl[3 * i + k];
      tot = fmaf(a.w_rot * dR[i][k], dR[i][k], tot);
    }
  }
  const float E[3][3] = {{R[0][0], R[0][1], R[0][2]}, {R[1][0], R[1][1], R[1][2]}, {R[2][0], R[2][1], R[2][2]}};
  const float te[3] = {t[0], t[1], t[2]};
  // joint axes again, with the path's collision gradient and the bounds
  const uint32_t* jrow = reinterpret_cast<const uint32_t*>(w.cjg + c * jstride);
  float Rc[3][3] = {{1.f, 0.f, 0.f}, {0.f, 1.f, 0.f}, {0.f, 0.f, 1.f}}, tc[3] = {0.f, 0.f, 0.f};
  for (int j = 0; j < J; ++j) {
    chain_step(a.joint_fixed + 12 * j, qc[j], Rc, tc);
    const float ax = Rc[0][2], ay = Rc[1][2], az = Rc[2][2];  // z axis of T_j
    const float rx = te[0] - tc[0], ry = te[1] - tc[1], rz = te[2] - tc[2];
    float gj = 2.f * a.w_pos *
               (dt[0] * (ay * rz - az * ry) + dt[1] * (az * rx - ax * rz) + dt[2] * (ax * ry - ay * rx));
#pragma unroll
    for (int k = 0; k < 3; ++k) {  // column k of R turns as a x R_k
      const float vx = ay * E[2][k] - az * E[1][k], vy = az * E[0][k] - ax * E[2][k],
                  vz = ax * E[1][k] - ay * E[0][k];
      gj = fmaf(2.f * a.w_rot, dR[0][k] * vx + dR[1][k] * vy + dR[2][k] * vz, gj);
    }
    const float qj = qc[j], hi = a.q_hi[j], lo = a.q_lo[j];
    if (qj > hi) {
      tot = fmaf(a.w_bound * (qj - hi), qj - hi, tot);
      gj = fmaf(2.f * a.w_bound, qj - hi, gj);
    } else if (qj < lo) {
      tot = fmaf(a.w_bound * (lo - qj), lo - qj, tot);
      gj = fmaf(-2.f * a.w_bound, lo - qj, gj);
    }
    const int wd = j / fj.k;
    w.cgrad[c * J + j] = unpack_slot(jrow[wd], j - wd * fj.k, fj) + gj;
  }
  w.ctot[c] = tot;
}

// Steepest descent scaled so that the largest joint move is step0.
template <int JT>
__device__ __forceinline__ void restart_dir(const float* g, float* d, float step0) {
  float mx = 0.f;
#pragma unroll
  for (int j = 0; j < JT; ++j) mx = fmaxf(mx, fabsf(g[j]));
  const float s = mx > 0.f ? step0 / mx : 0.f;
#pragma unroll
  for (int j = 0; j < JT; ++j) d[j] = -g[j] * s;
}

// One thread per seed; JT = the arm's joint count at compile time, so the
// per-joint vectors live in registers.  init: candidates are the seeds
// themselves (N = 1) and nothing is compared.
template <int JT>
__global__ void __launch_bounds__(64) ik_update(IkArgs a, float* __restrict__ q, IkWork w,
                                                float* __restrict__ cost, int32_t* __restrict__ pick,
                                                int N, int init) {
  constexpr int J = JT;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const int m = a.m;
  int best = 0;
  float fb = w.ctot[i * N];
  for (int k = 1; k < N; ++k) {
    const float f = w.ctot[i * N + k];
    if (f < fb) {
      fb = f;
      best = k;
    }
  }
  const int64_t cb = i * N + best;
  float gn[J], qn[J];
#pragma unroll
  for (int j = 0; j < J; ++j) {
    gn[j] = w.cgrad[cb * J + j];
    qn[j] = w.cq[cb * J + j];
  }
  float* S = w.S + i * m * J;
  float* Y = w.Y + i * m * J;
  int cnt = init ? 0 : w.mcount[i];
  int head = init ? 0 : w.mhead[i];
  auto slot = [&](int k) {  // ring slot of pair k (0 = oldest)
    const int sl = head + k;
    return sl >= m ? sl - m : sl;
  };
  float* d = w.d + i * J;
  if (init || a.scales[best] == 0.f) {
    cnt = 0;
    head = 0;
    float dn[J];
    restart_dir<J>(gn, dn, a.step0);
#pragma unroll
    for (int j = 0; j < J; ++j) d[j] = dn[j];
  } else {
    float sy = 0.f;
#pragma unroll
    for (int j = 0; j < J; ++j) sy = fmaf(qn[j] - q[i * J + j], gn[j] - w.g[i * J + j], sy);
    if (sy > 0.f) {
      if (cnt == m) {  // drop the oldest pair
        head = head + 1 == m ? 0 : head + 1;
        --cnt;
      }
      const int sn = slot(cnt);
#pragma unroll
      for (int j = 0; j < J; ++j) {
        S[sn * J + j] = qn[j] - q[i * J + j];
        Y[sn * J + j] = gn[j] - w.g[i * J + j];
      }
      ++cnt;
    }
    float dd[J];
    if (cnt == 0) {
      restart_dir<J>(gn, dd, a.step0);
    } else {  // two-loop recursion, H0 = (s.y / y.y) I of the newest pair
      float alpha[VAPR_IK_MAX_HISTORY], rho[VAPR_IK_MAX_HISTORY];
#pragma unroll
      for (int j = 0; j < J; ++j) dd[j] = -gn[j];
#pragma unroll
      for (int k = VAPR_IK_MAX_HISTORY - 1; k >= 0; --k) {
        if (k >= cnt) continue;
        const float* Sk = S + slot(k) * J;
        const float* Yk = Y + slot(k) * J;
        float s_y = 0.f, s_q = 0.f;
#pragma unroll
        for (int j = 0; j < J; ++j) {
          s_y = fmaf(Sk[j], Yk[j], s_y);
          s_q = fmaf(Sk[j], dd[j], s_q);
        }
        rho[k] = 1.f / s_y;
        alpha[k] = rho[k] * s_q;
#pragma unroll
        for (int j = 0; j < J; ++j) dd[j] = fmaf(-alpha[k], Yk[j], dd[j]);
      }
      float s_y = 0.f, y_y = 0.f;
      const float* Sn = S + slot(cnt - 1) * J;
      const float* Yn = Y + slot(cnt - 1) * J;
#pragma unroll
      for (int j = 0; j < J; ++j) {
        s_y = fmaf(Sn[j], Yn[j], s_y);
        y_y = fmaf(Yn[j], Yn[j], y_y);
      }
      const float gam = s_y / y_y;
#pragma unroll
      for (int j = 0; j < J; ++j) dd[j] *= gam;
#pragma unroll
      for (int k = 0; k < VAPR_IK_MAX_HISTORY; ++k) {
        if (k >= cnt) continue;
        const float* Sk = S + slot(k) * J;
        const float* Yk = Y + slot(k) * J;
        float yr = 0.f;
#pragma unroll
        for (int j = 0; j < J; ++j) yr = fmaf(Yk[j], dd[j], yr);
        const float beta = rho[k] * yr;
#pragma unroll
        for (int j = 0; j < J; ++j) dd[j] = fmaf(alpha[k] - beta, Sk[j], dd[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < J; ++j) d[j] = dd[j];
  }
  w.mcount[i] = cnt;
  w.mhead[i] = head;
#pragma unroll
  for (int j = 0; j < J; ++j) {
    w.g[i * J + j] = gn[j];
    if (!init) q[i * J + j] = qn[j];
  }
  if (cost) cost[i] = fb;
  if (pick) pick[i] = best;
}

template <int JT>
static void launch_update_j(const IkArgs& a, float* q, const IkWork& w, float* cost, int32_t* pick, int N,
                            int init, cudaStream_t st) {
  ik_update<JT><<<(int)((a.n + 63) / 64), 64, 0, st>>>(a, q, w, cost, pick, N, init);
}

static void launch_update(const IkArgs& a, float* q, const IkWork& w, float* cost, int32_t* pick, int N,
                          int init, cudaStream_t st) {
  switch (a.J) {
#define VAPR_IK_J(n) \
  case n: launch_update_j<n>(a, q, w, cost, pick, N, init, st); break;
    VAPR_IK_J(1) VAPR_IK_J(2) VAPR_IK_J(3) VAPR_IK_J(4) VAPR_IK_J(5) VAPR_IK_J(6) VAPR_IK_J(7)
    VAPR_IK_J(8) VAPR_IK_J(9) VAPR_IK_J(10) VAPR_IK_J(11) VAPR_IK_J(12) VAPR_IK_J(13)
    VAPR_IK_J(14) VAPR_IK_J(15) VAPR_IK_J(16)
#undef VAPR_IK_J
    default: break;
  }
}

static vapr_status check_ik(const vapr_robot* robot, const vapr_scene* scene, const vapr_cost_params* params,
                            const vapr_ik_params* ik, const float* goal, const void* q, int64_t n,
                            const vapr_format_table* table, RobotArgs* r) {
  vapr_status v = check_robot(robot, r);
  if (v != VAPR_OK) return v;
  if ((v = check_table(table)) != VAPR_OK) return v;
  if (!params || !ik) return VAPR_ERR_INVALID_ARG;
  SceneArgs sc;
  if ((v = check_scene(scene, &sc)) != VAPR_OK) return v;
  if (ik->n_scales < 1 || ik->n_scales > VAPR_IK_MAX_SCALES || ik->history < 1 ||
      ik->history > VAPR_IK_MAX_HISTORY || !(ik->step0 > 0.f) || !ik->q_lo || !ik->q_hi)
    return VAPR_ERR_INVALID_ARG;
  if (n < 0) return VAPR_ERR_INVALID_ARG;
  if (n > VAPR_MAX_CONFIGS) return VAPR_ERR_TOO_LARGE;
  if (n > 0 && (!goal || !q)) return VAPR_ERR_INVALID_ARG;
  if ((uintptr_t)goal % 4 || (uintptr_t)q % 4) return VAPR_ERR_MISALIGNED;
  return VAPR_OK;
}

static IkArgs make_args(const RobotArgs& r, const vapr_ik_params* ik, const float* goal, int64_t n) {
  IkArgs a;
  a.J = r.J;
  a.N = ik->n_scales;
  a.m = ik->history;
  a.n = n;
  a.w_pos = ik->w_pos;
  a.w_rot = ik->w_rot;
  a.w_bound = ik->w_bound;
  a.step0 = ik->step0;
  for (int k = 0; k < VAPR_IK_MAX_SCALES; ++k) a.scales[k] = k < ik->n_scales ? ik->scales[k] : 0.f;
  a.q_lo = ik->q_lo;
  a.q_hi = ik->q_hi;
  a.joint_fixed = r.joint_fixed;
  a.goal = goal;
  return a;
}

// Candidates -> path -> terms -> update, with N candidates per seed.
static cudaError_t run_iteration(const RobotArgs& r, const vapr_scene* scene, const vapr_cost_params* p,
                                 IkArgs a, const vapr_format_table* t, IkWork& w, float* q, float* cost,
                                 int32_t* pick, int N, bool init, cudaStream_t st) {
  const int64_t c = a.n * N;
  cudaError_t e;
  if (init) {
    e = cudaMemcpyAsync(w.cq, q, (size_t)a.n * r.J * 4, cudaMemcpyDeviceToDevice, st);
  } else {
    ik_candidates<<<(int)((c + 255) / 256), 256, 0, st>>>(a, q, w, N);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return e;
  SceneArgs sc;
  check_scene(scene, &sc);  // checked by the entry point
  Packed none{nullptr, 0, make_dev_fmt(t->xform)};
  Packed P{w.path, (int64_t)row_bytes(3 * (int64_t)r.S, t->pos), make_dev_fmt(t->pos)};
  Packed G{w.path + w.P_bytes, (int64_t)row_bytes(3 * (int64_t)r.S, t->grad), make_dev_fmt(t->grad)};
  Packed D{nullptr, 0, make_dev_fmt(t->dist)};
  Packed Jg{w.cjg, (int64_t)row_bytes(r.J, t->jgrad), make_dev_fmt(t->jgrad)};
  if ((e = launch_fk(r, w.cq, c, P, none, st)) != cudaSuccess) return e;
  if ((e = launch_collision(r, sc, *p, P, c, w.ccoll, D, G, st)) != cudaSuccess) return e;
  if ((e = launch_backward(r, w.cq, none, G, nullptr, c, Jg, st)) != cudaSuccess) return e;
  ik_terms<<<(int)((c + 127) / 128), 128, 0, st>>>(a, w, Jg.f, Jg.stride, N);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  launch_update(a, q, w, cost, pick, N, init ? 1 : 0, st);
  return cudaGetLastError();
}

}  // namespace vapr

using namespace vapr;

extern "C" size_t vapr_ik_workspace_bytes(const vapr_robot* robot, int64_t n_seeds, const vapr_ik_params* ik,
                                          const vapr_format_table* table) {
  RobotArgs r;
  if (check_robot(robot, &r) != VAPR_OK || check_table(table) != VAPR_OK || !ik || n_seeds < 0 ||
      ik->n_scales < 1 || ik->n_scales > VAPR_IK_MAX_SCALES || ik->history < 1 ||
      ik->history > VAPR_IK_MAX_HISTORY)
    return 0;
  return carve_ik(nullptr, r, n_seeds, ik->n_scales, ik->history, table).bytes;
}

extern "C" vapr_status vapr_ik_init(const vapr_robot* robot, const vapr_scene* scene,
                                    const vapr_cost_params* params, const vapr_ik_params* ik, const float* goal,
                                    const float* q, int64_t n_seeds, const vapr_format_table* table,
                                    void* workspace, size_t workspace_bytes, float* cost, void* stream) {
  RobotArgs r;
  vapr_status v = check_ik(robot, scene, params, ik, goal, q, n_seeds, table, &r);
  if (v != VAPR_OK) return v;
  if (n_seeds == 0) return VAPR_OK;
  if (!workspace || (uintptr_t)workspace % 256) return workspace ? VAPR_ERR_MISALIGNED : VAPR_ERR_INVALID_ARG;
  IkWork w = carve_ik(workspace, r, n_seeds, ik->n_scales, ik->history, table);
  if (workspace_bytes < w.bytes) return VAPR_ERR_INVALID_ARG;
  IkArgs a = make_args(r, ik, goal, n_seeds);
  a.scales[0] = 0.f;
  return cuda_status(run_iteration(r, scene, params, a, table, w, const_cast<float*>(q), cost, nullptr, 1, true,
                                   (cudaStream_t)stream));
}

extern "C" vapr_status vapr_ik_step(const vapr_robot* robot, const vapr_scene* scene,
                                    const vapr_cost_params* params, const vapr_ik_params* ik, const float* goal,
                                    float* q, int64_t n_seeds, const vapr_format_table* table, void* workspace,
                                    size_t workspace_bytes, float* cost, int32_t* pick, void* stream) {
  RobotArgs r;
  vapr_status v = check_ik(robot, scene, params, ik, goal, q, n_seeds, table, &r);
  if (v != VAPR_OK) return v;
  if (n_seeds == 0) return VAPR_OK;
  if (!workspace || (uintptr_t)workspace % 256) return workspace ? VAPR_ERR_MISALIGNED : VAPR_ERR_INVALID_ARG;
  IkWork w = carve_ik(workspace, r, n_seeds, ik->n_scales, ik->history, table);
  if (workspace_bytes < w.bytes) return VAPR_ERR_INVALID_ARG;
  if (n_seeds * ik->n_scales > ((int64_t)1 << 31)) return VAPR_ERR_TOO_LARGE;
  return cuda_status(run_iteration(r, scene, params, make_args(r, ik, goal, n_seeds), table, w, q, cost, pick,
                                   ik->n_scales, false, (cudaStream_t)stream));
}
