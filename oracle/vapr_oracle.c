/*
 * FP64 CPU oracle for the VaPr batched cost-and-gradient path.
 * TEST INFRASTRUCTURE ONLY (see vapr_oracle.h): plain loops in double
 * precision, one configuration at a time, no blocking or fusion.
 */
#include "vapr_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the later parallel loops (n >= 1); the arithmetic of each
 * configuration does not depend on it. */
void or_set_num_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ========================================================================= */
/* ExMy emulator.  Sec. IV-A: a format has 1 sign bit, E exponent bits and M
 * mantissa bits.  Reading: IEEE-style bias 2^(E-1)-1 with subnormals; the
 * conversion rounds to nearest, ties to even (Sec. V-B names the "_rn"
 * intrinsics), in the subnormal range too; signed zero is kept.  E8M23 is
 * float32 itself and passes through unchanged. */

static int is_identity(int E, int M) { return E == 8 && M == 23; }

typedef struct {
  int E, M, bias, emin;      /* emin: exponent of the smallest normal */
  uint32_t all_e, all_m;     /* all-ones exponent / mantissa fields */
  uint32_t max_code;         /* largest finite magnitude */
  uint32_t inf_code;         /* Inf magnitude (IEEE only) */
  uint32_t nan_code;         /* code produced for a NaN input */
  double max_val;
  int overflow_to_inf;       /* IEEE without SAT */
} or_fmt;

static or_fmt fmt_info(int E, int M, unsigned flags) {
  or_fmt f;
  f.E = E;
  f.M = M;
  f.bias = (1 << (E - 1)) - 1;
  f.emin = 1 - f.bias;
  f.all_e = (1u << E) - 1u;
  f.all_m = (1u << M) - 1u;
  uint32_t emax_field, mmax;
  if (flags & OR_IEEE) {
    emax_field = f.all_e - 1u;
    mmax = f.all_m;
  } else if (flags & OR_FN) {
    emax_field = f.all_e;
    mmax = f.all_m - 1u;
  } else {
    emax_field = f.all_e;
    mmax = f.all_m;
  }
  f.max_code = (emax_field << M) | mmax;
  f.max_val = ldexp(1.0 + (double)mmax / ldexp(1.0, M), (int)emax_field - f.bias);
  f.inf_code = f.all_e << M;
  /* NaN input: the canonical positive NaN (all-ones exponent and mantissa)
   * where the format has NaN; otherwise the largest positive finite value. */
  f.nan_code = (flags & (OR_IEEE | OR_FN)) ? ((f.all_e << M) | f.all_m) : f.max_code;
  f.overflow_to_inf = (flags & OR_IEEE) && !(flags & OR_SAT);
  return f;
}

double or_exmy_max_finite(int E, int M, unsigned flags) {
  if (is_identity(E, M)) return 3.4028234663852886e38;
  return fmt_info(E, M, flags).max_val;
}

uint32_t or_exmy_encode(float xf, int E, int M, unsigned flags) {
  if (is_identity(E, M)) {
    uint32_t u;
    memcpy(&u, &xf, 4);
    return u;
  }
  or_fmt f = fmt_info(E, M, flags);
  double x = (double)xf;
  if (isnan(x)) return f.nan_code;
  uint32_t s = signbit(x) ? (1u << (E + M)) : 0u;
  double a = fabs(x);
  if (isinf(a)) return s | (f.overflow_to_inf ? f.inf_code : f.max_code);
  if (a == 0.0) return s;

  /* Round a to the format's grid.  Within binade [2^e, 2^(e+1)) the spacing
   * is 2^(e-M); below the smallest normal it stays 2^(emin-M).  The exponent
   * is left unbounded above so that overflow is decided on the rounded
   * value, as IEEE round-to-nearest does. */
  int e2;
  frexp(a, &e2); /* a = f * 2^e2, f in [0.5, 1) */
  int e = e2 - 1;
  int quantum_exp = (e < f.emin ? f.emin : e) - M;
  double n = nearbyint(ldexp(a, -quantum_exp)); /* exact scaling; RNE */
  double v = ldexp(n, quantum_exp);
  if (v > f.max_val) return s | (f.overflow_to_inf ? f.inf_code : f.max_code);
  if (v == 0.0) return s;

  if (v < ldexp(1.0, f.emin)) /* subnormal: exponent field 0 */
    return s | (uint32_t)ldexp(v, M - f.emin);
  frexp(v, &e2);
  e = e2 - 1;
  uint32_t mant = (uint32_t)(ldexp(v, M - e) - ldexp(1.0, M));
  return s | ((uint32_t)(e + f.bias) << M) | mant;
}

double or_exmy_decode(uint32_t code, int E, int M, unsigned flags) {
  if (is_identity(E, M)) {
    float x;
    memcpy(&x, &code, 4);
    return (double)x;
  }
  or_fmt f = fmt_info(E, M, flags);
  double sign = ((code >> (E + M)) & 1u) ? -1.0 : 1.0;
  uint32_t ef = (code >> M) & f.all_e;
  uint32_t mf = code & f.all_m;
  if ((flags & OR_IEEE) && ef == f.all_e) return mf ? NAN : sign * INFINITY;
  if ((flags & OR_FN) && ef == f.all_e && mf == f.all_m) return NAN;
  if (ef == 0) return sign * ldexp((double)mf, f.emin - M);
  return sign * ldexp(1.0 + (double)mf / ldexp(1.0, M), (int)ef - f.bias);
}

void or_exmy_encode_batch(const float* x, int64_t n, int E, int M,
                          unsigned flags, uint32_t* codes) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) codes[i] = or_exmy_encode(x[i], E, M, flags);
}

void or_exmy_encode_bits_range(uint32_t start, int64_t count, int E, int M,
                               unsigned flags, uint32_t* codes) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < count; ++i) {
    uint32_t u = start + (uint32_t)i;
    float x;
    memcpy(&x, &u, 4);
    codes[i] = or_exmy_encode(x, E, M, flags);
  }
}

void or_exmy_decode_batch(const uint32_t* codes, int64_t n, int E, int M,
                          unsigned flags, double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) out[i] = or_exmy_decode(codes[i], E, M, flags);
}

/* Sec. IV-A: one 32-bit register holds floor(32/bits) values. */
void or_pack_rows(const uint32_t* codes, int64_t rows, int64_t row_len,
                  int bits, uint8_t* dst, int64_t row_stride_bytes) {
  int k = 32 / bits;
  uint32_t mask = bits == 32 ? 0xffffffffu : ((1u << bits) - 1u);
  for (int64_t r = 0; r < rows; ++r) {
    uint8_t* row = dst + r * row_stride_bytes;
    memset(row, 0, (size_t)row_stride_bytes);
    for (int64_t i = 0; i < row_len; ++i) {
      int64_t w = i / k;
      int sh = bits * (int)(i % k);
      uint32_t word;
      memcpy(&word, row + 4 * w, 4);
      word |= (codes[r * row_len + i] & mask) << sh;
      memcpy(row + 4 * w, &word, 4);
    }
  }
}

void or_unpack_rows(const uint8_t* src, int64_t rows, int64_t row_len,
                    int bits, int64_t row_stride_bytes, uint32_t* codes) {
  int k = 32 / bits;
  uint32_t mask = bits == 32 ? 0xffffffffu : ((1u << bits) - 1u);
  for (int64_t r = 0; r < rows; ++r) {
    const uint8_t* row = src + r * row_stride_bytes;
    for (int64_t i = 0; i < row_len; ++i) {
      uint32_t word;
      memcpy(&word, row + 4 * (i / k), 4);
      codes[r * row_len + i] = (word >> (bits * (int)(i % k))) & mask;
    }
  }
}

/* ========================================================================= */
/* Kinematics with 4x4 homogeneous matrices, row-major. */

static void mat4_identity(double A[16]) {
  memset(A, 0, 16 * sizeof(double));
  A[0] = A[5] = A[10] = A[15] = 1.0;
}

static void mat4_mul(const double A[16], const double B[16], double C[16]) {
  double T[16];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double acc = 0.0;
      for (int k = 0; k < 4; ++k) acc += A[4 * i + k] * B[4 * k + j];
      T[4 * i + j] = acc;
    }
  memcpy(C, T, sizeof(T));
}

/* 3x4 table row (R row-major, then t) -> 4x4 */
static void mat4_from_3x4(const float* m, double A[16]) {
  mat4_identity(A);
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) A[4 * i + j] = (double)m[3 * i + j];
    A[4 * i + 3] = (double)m[9 + i];
  }
}

static void mat4_rot_z(double q, double A[16]) {
  mat4_identity(A);
  A[0] = cos(q);
  A[1] = -sin(q);
  A[4] = sin(q);
  A[5] = cos(q);
}

/* all link transforms T_1..T_nj of one configuration, 4x4 each */
static void chain(int nj, const float* joint_fixed, const float* q, double* T) {
  double prev[16], F[16], Rz[16], A[16];
  mat4_identity(prev);
  for (int i = 0; i < nj; ++i) {
    mat4_from_3x4(joint_fixed + 12 * i, F);
    mat4_rot_z((double)q[i], Rz);
    mat4_mul(F, Rz, A);
    mat4_mul(prev, A, T + 16 * i);
    memcpy(prev, T + 16 * i, sizeof(prev));
  }
}

static void apply(const double A[16], const double p[3], double out[3]) {
  for (int i = 0; i < 3; ++i)
    out[i] = A[4 * i] * p[0] + A[4 * i + 1] * p[1] + A[4 * i + 2] * p[2] + A[4 * i + 3];
}

void or_fk(int nj, const float* joint_fixed, int ns, const float* sphere_local,
           const int32_t* sphere_link, const float* q, int64_t n,
           double* xform, double* pos) {
#pragma omp parallel
  {
    double* T = (double*)malloc(sizeof(double) * 16 * (size_t)nj);
#pragma omp for schedule(static)
    for (int64_t c = 0; c < n; ++c) {
      chain(nj, joint_fixed, q + (int64_t)nj * c, T);
      if (xform) {
        for (int i = 0; i < nj; ++i) {
          double* out = xform + ((int64_t)nj * c + i) * 12;
          for (int r = 0; r < 3; ++r) {
            for (int k = 0; k < 3; ++k) out[3 * r + k] = T[16 * i + 4 * r + k];
            out[9 + r] = T[16 * i + 4 * r + 3];
          }
        }
      }
      for (int s = 0; s < ns; ++s) {
        double p[3] = {sphere_local[4 * s], sphere_local[4 * s + 1], sphere_local[4 * s + 2]};
        apply(T + 16 * (sphere_link[s] - 1), p, pos + ((int64_t)ns * c + s) * 3);
      }
    }
    free(T);
  }
}

/* ========================================================================= */
/* Oriented-box signed distance.  x = R^T (c - t), u = |x| - h,
 * d = |max(u, 0)| + min(max_k u_k, 0).  Gradient (world frame): outside,
 * R (sgn(x) * max(u, 0)) / |max(u, 0)|; inside or on the surface,
 * R sgn(x_k) e_k with k = argmax_k u_k (lowest k on ties, sgn(0) = +1).
 * *branch_margin receives the distance to the nearest gradient
 * discontinuity: the top-two gap of u and |x_k| inside, +inf outside. */
static double box_sdf(const float* pose, const float* half, const double c[3],
                      double grad[3], double* branch_margin) {
  double R[9], t[3], h[3], x[3], u[3], gl[3];
  for (int i = 0; i < 9; ++i) R[i] = pose[i];
  for (int i = 0; i < 3; ++i) {
    t[i] = pose[9 + i];
    h[i] = half[i];
  }
  for (int k = 0; k < 3; ++k) {
    x[k] = 0.0;
    for (int i = 0; i < 3; ++i) x[k] += R[3 * i + k] * (c[i] - t[i]);
    u[k] = fabs(x[k]) - h[k];
  }
  double d;
  int outside = u[0] > 0.0 || u[1] > 0.0 || u[2] > 0.0;
  if (outside) {
    double v[3], nrm = 0.0;
    for (int k = 0; k < 3; ++k) {
      v[k] = u[k] > 0.0 ? u[k] : 0.0;
      nrm += v[k] * v[k];
    }
    nrm = sqrt(nrm);
    d = nrm;
    for (int k = 0; k < 3; ++k) gl[k] = (x[k] >= 0.0 ? 1.0 : -1.0) * v[k] / nrm;
    *branch_margin = INFINITY;
  } else {
    int ks = 0;
    for (int k = 1; k < 3; ++k)
      if (u[k] > u[ks]) ks = k;
    d = u[ks];
    double gap = INFINITY;
    for (int k = 0; k < 3; ++k)
      if (k != ks && u[ks] - u[k] < gap) gap = u[ks] - u[k];
    *branch_margin = fmin(gap, fabs(x[ks]));
    for (int k = 0; k < 3; ++k) gl[k] = 0.0;
    gl[ks] = x[ks] >= 0.0 ? 1.0 : -1.0;
  }
  for (int i = 0; i < 3; ++i) grad[i] = R[3 * i] * gl[0] + R[3 * i + 1] * gl[1] + R[3 * i + 2] * gl[2];
  return d;
}

void or_box_sdf_batch(const float* pose, const float* half, const double* pts,
                      int64_t m, double* d, double* grad) {
  for (int64_t i = 0; i < m; ++i) {
    double margin;
    d[i] = box_sdf(pose + 12 * i, half + 3 * i, pts + 3 * i, grad + 3 * i, &margin);
  }
}

void or_scene_sdf(int no, const float* pose, const float* half,
                  const double* pts, int64_t m, double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < m; ++i) {
    double best = INFINITY, g[3], margin;
    for (int o = 0; o < no; ++o) {
      double d = box_sdf(pose + 12 * o, half + 3 * o, pts + 3 * i, g, &margin);
      if (d < best) best = d;
    }
    out[i] = best;
  }
}

/* ========================================================================= */
/* Collision cost and its gradient with respect to the sphere centres.
 * Reading: the environment term sums the hinge over all cuboids (the paper
 * does not say sum, min or max); the hinge's subgradient at exactly zero
 * penetration is 0; a self pair at zero distance contributes no gradient. */
void or_collision(int ns, const float* sphere_local, int npairs,
                  const int32_t* pairs, int no, const float* pose,
                  const float* half, double eta, double eta_s, double w_c,
                  double w_s, const double* pos, int64_t n, double* cost,
                  double* dist, double* grad, int32_t* kink, double kink_eps) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t c = 0; c < n; ++c) {
    const double* P = pos + (int64_t)ns * 3 * c;
    double* G = grad + (int64_t)ns * 3 * c;
    int32_t* K = kink ? kink + (int64_t)ns * c : NULL;
    double total = 0.0;
    for (int s = 0; s < ns; ++s) {
      double r = sphere_local[4 * s + 3];
      double Ds = 0.0, gs[3] = {0.0, 0.0, 0.0};
      int flag = 0;
      for (int o = 0; o < no; ++o) {
        double gd[3], margin;
        double d = box_sdf(pose + 12 * o, half + 3 * o, P + 3 * s, gd, &margin);
        double pen = r + eta - d;
        if (fabs(pen) < kink_eps) flag = 1;
        if (pen > 0.0) {
          Ds += pen;
          for (int k = 0; k < 3; ++k) gs[k] -= gd[k];
          if (margin < kink_eps) flag = 1;
        }
      }
      dist[(int64_t)ns * c + s] = Ds;
      for (int k = 0; k < 3; ++k) G[3 * s + k] = w_c * gs[k];
      total += w_c * Ds;
      if (K) K[s] = flag;
    }
    for (int p = 0; p < npairs; ++p) {
      int i = pairs[2 * p], j = pairs[2 * p + 1];
      double diff[3], d2 = 0.0;
      for (int k = 0; k < 3; ++k) {
        diff[k] = P[3 * i + k] - P[3 * j + k];
        d2 += diff[k] * diff[k];
      }
      double dd = sqrt(d2);
      double pen = (double)sphere_local[4 * i + 3] + (double)sphere_local[4 * j + 3] + eta_s - dd;
      if (K && (fabs(pen) < kink_eps || (pen > 0.0 && dd < kink_eps))) K[i] = K[j] = 1;
      if (pen > 0.0) {
        total += w_s * pen;
        if (dd > 0.0) {
          for (int k = 0; k < 3; ++k) {
            G[3 * i + k] -= w_s * diff[k] / dd;
            G[3 * j + k] += w_s * diff[k] / dd;
          }
        }
      }
    }
    cost[c] = total;
  }
}

/* ========================================================================= */
/* Backward kinematics: dc_s/dq_j = a_j x (c_s - o_j) for every sphere on a
 * link at or beyond joint j (a revolute joint turns everything after it),
 * so dC/dq_j = sum_s G_s . (a_j x (c_s - o_j)). */
/* Hinge sum over the cuboids at point x for a sphere of radius r: returns
 * sum_o max(0, r + eta - d_o(x)) and adds -grad of it to g; sets *kink when
 * x is within kink_eps of a hinge activation or, where active, of an
 * inside-argmax tie. */
static double hinge_sum(int no, const float* pose, const float* half, double r, double eta,
                        const double x[3], double g[3], int* kink, double kink_eps) {
  double D = 0.0;
  for (int o = 0; o < no; ++o) {
    double gd[3], margin;
    const double d = box_sdf(pose + 12 * o, half + 3 * o, x, gd, &margin);
    const double pen = r + eta - d;
    if (fabs(pen) < kink_eps) *kink = 1;
    if (pen > 0.0) {
      D += pen;
      for (int k = 0; k < 3; ++k) g[k] -= gd[k];
      if (margin < kink_eps) *kink = 1;
    }
  }
  return D;
}

void or_swept(int ns, const float* sphere_local, int no, const float* pose, const float* half,
              double eta, double w_c, const double* pos, int64_t n, int horizon, int samples,
              double* cost, double* dist, double* grad, int32_t* kink, double kink_eps) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t c = 0; c < n; ++c) {
    const int h = (int)(c % horizon);
    const int64_t nxt = h + 1 < horizon ? c + 1 : c;  /* the row this one sweeps toward */
    const double* P = pos + (int64_t)ns * 3 * c;
    const double* Pn = pos + (int64_t)ns * 3 * nxt;
    const double* Pp = h > 0 ? pos + (int64_t)ns * 3 * (c - 1) : NULL;  /* sweeps toward c */
    double total = 0.0;
    for (int s = 0; s < ns; ++s) {
      const double r = sphere_local[4 * s + 3];
      double Ds = 0.0, gs[3] = {0.0, 0.0, 0.0};
      int flag = 0;
      for (int k = 0; k < samples; ++k) {
        const double a = (double)k / (double)samples;
        double x[3], g[3] = {0.0, 0.0, 0.0};
        /* own points: weight (1 - a), plus a when the row sweeps toward itself */
        for (int i = 0; i < 3; ++i) x[i] = (1.0 - a) * P[3 * s + i] + a * Pn[3 * s + i];
        Ds += hinge_sum(no, pose, half, r, eta, x, g, &flag, kink_eps);
        const double wown = nxt == c ? 1.0 : 1.0 - a;
        for (int i = 0; i < 3; ++i) gs[i] += wown * g[i];
        /* the previous row's points depend on this row with weight a */
        if (Pp && a > 0.0) {
          double gp[3] = {0.0, 0.0, 0.0};
          for (int i = 0; i < 3; ++i) x[i] = (1.0 - a) * Pp[3 * s + i] + a * P[3 * s + i];
          hinge_sum(no, pose, half, r, eta, x, gp, &flag, kink_eps);
          for (int i = 0; i < 3; ++i) gs[i] += a * gp[i];
        }
      }
      dist[(int64_t)ns * c + s] = Ds;
      for (int i = 0; i < 3; ++i) grad[(int64_t)ns * 3 * c + 3 * s + i] = w_c * gs[i];
      total += w_c * Ds;
      if (kink) kink[(int64_t)ns * c + s] = flag;
    }
    cost[c] = total;
  }
}

void or_backward(int nj, const float* joint_fixed, int ns,
                 const float* sphere_local, const int32_t* sphere_link,
                 const float* q, const double* grad, const double* dcost,
                 int64_t n, double* jgrad) {
#pragma omp parallel
  {
    double* T = (double*)malloc(sizeof(double) * 16 * (size_t)nj);
#pragma omp for schedule(static)
    for (int64_t c = 0; c < n; ++c) {
      chain(nj, joint_fixed, q + (int64_t)nj * c, T);
      double scale = dcost ? dcost[c] : 1.0;
      for (int j = 0; j < nj; ++j) {
        const double* Tj = T + 16 * j;
        double a[3] = {Tj[2], Tj[6], Tj[10]};  /* z column */
        double o[3] = {Tj[3], Tj[7], Tj[11]};  /* origin */
        double acc = 0.0;
        for (int s = 0; s < ns; ++s) {
          if (sphere_link[s] - 1 < j) continue;
          double p[3] = {sphere_local[4 * s], sphere_local[4 * s + 1], sphere_local[4 * s + 2]};
          double cs[3], rel[3], dc[3];
          apply(T + 16 * (sphere_link[s] - 1), p, cs);
          for (int k = 0; k < 3; ++k) rel[k] = cs[k] - o[k];
          dc[0] = a[1] * rel[2] - a[2] * rel[1];
          dc[1] = a[2] * rel[0] - a[0] * rel[2];
          dc[2] = a[0] * rel[1] - a[1] * rel[0];
          const double* g = grad + ((int64_t)ns * c + s) * 3;
          acc += g[0] * dc[0] + g[1] * dc[1] + g[2] * dc[2];
        }
        jgrad[(int64_t)nj * c + j] = scale * acc;
      }
    }
    free(T);
  }
}

/* ========================================================================= */
/* Surrogate network: a plain forward pass and the chain rule, one sample at
 * a time. */

static double silu(double z) { return z / (1.0 + exp(-z)); }
static double silu_grad(double z) {
  const double sg = 1.0 / (1.0 + exp(-z));
  return sg * (1.0 + z * (1.0 - sg));
}

typedef struct {
  const float *W1, *b1, *W2, *b2, *W3, *b3, *w4, *b4;
} or_net;

static or_net net_view(const float* p, int H) {
  or_net v;
  v.W1 = p;
  v.b1 = v.W1 + 3 * H;
  v.W2 = v.b1 + H;
  v.b2 = v.W2 + H * H;
  v.W3 = v.b2 + H;
  v.b3 = v.W3 + H * H;
  v.w4 = v.b3 + H;
  v.b4 = v.w4 + H;
  return v;
}

/* z1..z3 and a1..a3 of one sample (each length H); returns f */
static double net_eval(const or_net* v, int H, const float* x, double* z1, double* a1, double* z2,
                       double* a2, double* z3, double* a3) {
  for (int i = 0; i < H; ++i) {
    z1[i] = v->b1[i];
    for (int k = 0; k < 3; ++k) z1[i] += (double)v->W1[3 * i + k] * x[k];
    a1[i] = silu(z1[i]);
  }
  for (int i = 0; i < H; ++i) {
    z2[i] = v->b2[i];
    for (int k = 0; k < H; ++k) z2[i] += (double)v->W2[(int64_t)H * i + k] * a1[k];
    a2[i] = silu(z2[i]);
  }
  for (int i = 0; i < H; ++i) {
    z3[i] = v->b3[i];
    for (int k = 0; k < H; ++k) z3[i] += (double)v->W3[(int64_t)H * i + k] * a2[k];
    a3[i] = silu(z3[i]);
  }
  double f = v->b4[0];
  for (int i = 0; i < H; ++i) f += (double)v->w4[i] * a3[i];
  return f;
}

static double round_bf16(double v) {
  return or_exmy_decode(or_exmy_encode((float)v, 8, 7, OR_IEEE), 8, 7, OR_IEEE);
}

void or_mlp_forward_bf16act(const float* params, int H, const float* x, int64_t n, double* out) {
  or_net v = net_view(params, H);
#pragma omp parallel
  {
    double* a1 = (double*)malloc(sizeof(double) * 2 * (size_t)H);
    double* a2 = a1 + H;
#pragma omp for schedule(static)
    for (int64_t s = 0; s < n; ++s) {
      const float* xs = x + 3 * s;
      for (int i = 0; i < H; ++i) {
        double z = v.b1[i];
        for (int k = 0; k < 3; ++k) z += (double)v.W1[3 * i + k] * xs[k];
        a1[i] = round_bf16(silu(z));
      }
      for (int i = 0; i < H; ++i) {
        double z = v.b2[i];
        for (int k = 0; k < H; ++k) z += (double)v.W2[(int64_t)H * i + k] * a1[k];
        a2[i] = round_bf16(silu(z));
      }
      double f = v.b4[0];
      for (int i = 0; i < H; ++i) {
        double z = v.b3[i];
        for (int k = 0; k < H; ++k) z += (double)v.W3[(int64_t)H * i + k] * a2[k];
        f += (double)v.w4[i] * silu(z);
      }
      out[s] = f;
    }
    free(a1);
  }
}

void or_mlp_forward(const float* params, int H, const float* x, int64_t n, double* out) {
  or_net v = net_view(params, H);
#pragma omp parallel
  {
    double* buf = (double*)malloc(sizeof(double) * 6 * (size_t)H);
#pragma omp for schedule(static)
    for (int64_t i = 0; i < n; ++i)
      out[i] = net_eval(&v, H, x + 3 * i, buf, buf + H, buf + 2 * H, buf + 3 * H, buf + 4 * H,
                        buf + 5 * H);
    free(buf);
  }
}

double or_mlp_grads(const float* params, int H, const float* x, const float* y, int64_t n,
                    double over_weight, double* grads) {
  or_net v = net_view(params, H);
  const int64_t P = 2 * (int64_t)H * H + 7 * (int64_t)H + 1;
  for (int64_t i = 0; i < P; ++i) grads[i] = 0.0;
  double* gW1 = grads;
  double* gb1 = gW1 + 3 * H;
  double* gW2 = gb1 + H;
  double* gb2 = gW2 + (int64_t)H * H;
  double* gW3 = gb2 + H;
  double* gb3 = gW3 + (int64_t)H * H;
  double* gw4 = gb3 + H;
  double* gb4 = gw4 + H;
  double* buf = (double*)malloc(sizeof(double) * 9 * (size_t)H);
  double *z1 = buf, *a1 = buf + H, *z2 = buf + 2 * H, *a2 = buf + 3 * H, *z3 = buf + 4 * H,
         *a3 = buf + 5 * H, *d3 = buf + 6 * H, *d2 = buf + 7 * H, *d1 = buf + 8 * H;
  double loss = 0.0;
  for (int64_t s = 0; s < n; ++s) {
    const float* xs = x + 3 * s;
    const double f = net_eval(&v, H, xs, z1, a1, z2, a2, z3, a3);
    const double r = f - (double)y[s];
    const double wt = r > 0.0 ? over_weight : 1.0;
    loss += wt * r * r / (double)n;
    const double df = 2.0 * wt * r / (double)n;  /* dL/df */
    gb4[0] += df;
    for (int i = 0; i < H; ++i) {
      gw4[i] += df * a3[i];
      d3[i] = df * v.w4[i] * silu_grad(z3[i]); /* dL/dz3 */
    }
    for (int i = 0; i < H; ++i) {
      gb3[i] += d3[i];
      for (int k = 0; k < H; ++k) gW3[(int64_t)H * i + k] += d3[i] * a2[k];
    }
    for (int k = 0; k < H; ++k) { /* dL/dz2 = (W3^T d3) * s'(z2) */
      double acc = 0.0;
      for (int i = 0; i < H; ++i) acc += (double)v.W3[(int64_t)H * i + k] * d3[i];
      d2[k] = acc * silu_grad(z2[k]);
    }
    for (int i = 0; i < H; ++i) {
      gb2[i] += d2[i];
      for (int k = 0; k < H; ++k) gW2[(int64_t)H * i + k] += d2[i] * a1[k];
    }
    for (int k = 0; k < H; ++k) { /* dL/dz1 = (W2^T d2) * s'(z1) */
      double acc = 0.0;
      for (int i = 0; i < H; ++i) acc += (double)v.W2[(int64_t)H * i + k] * d2[i];
      d1[k] = acc * silu_grad(z1[k]);
    }
    for (int i = 0; i < H; ++i) {
      gb1[i] += d1[i];
      for (int k = 0; k < 3; ++k) gW1[3 * i + k] += d1[i] * xs[k];
    }
  }
  free(buf);
  return loss;
}

/* ========================================================================= */
/* IK optimisation: total cost, gradient, and the L-BFGS direction. */

void or_ik_costs(int nj, const float* joint_fixed, int ns, const float* sphere_local,
                 const int32_t* sphere_link, int npairs, const int32_t* pairs, int no,
                 const float* pose, const float* half, double eta, double eta_s, double w_c,
                 double w_s, double w_pos, double w_rot, double w_bound, const float* q_lo,
                 const float* q_hi, const float* goal, const float* q, int64_t n, double* cost,
                 double* grad) {
  double* pos = (double*)malloc(sizeof(double) * 3 * (size_t)ns * (size_t)n);
  double* ccost = (double*)malloc(sizeof(double) * (size_t)n);
  double* dist = (double*)malloc(sizeof(double) * (size_t)ns * (size_t)n);
  double* g = (double*)malloc(sizeof(double) * 3 * (size_t)ns * (size_t)n);
  or_fk(nj, joint_fixed, ns, sphere_local, sphere_link, q, n, NULL, pos);
  or_collision(ns, sphere_local, npairs, pairs, no, pose, half, eta, eta_s, w_c, w_s, pos, n, ccost,
               dist, g, NULL, 0.0);
  or_backward(nj, joint_fixed, ns, sphere_local, sphere_link, q, g, NULL, n, grad);
#pragma omp parallel
  {
    double* T = (double*)malloc(sizeof(double) * 16 * (size_t)nj);
#pragma omp for schedule(static)
    for (int64_t c = 0; c < n; ++c) {
      const float* qc = q + (int64_t)nj * c;
      const float* gl = goal + 12 * c;
      chain(nj, joint_fixed, qc, T);
      const double* E = T + 16 * (nj - 1);
      double dt[3], dR[9], total = ccost[c];
      for (int i = 0; i < 3; ++i) dt[i] = E[4 * i + 3] - (double)gl[9 + i];
      for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) dR[3 * i + k] = E[4 * i + k] - (double)gl[3 * i + k];
      for (int i = 0; i < 3; ++i) total += w_pos * dt[i] * dt[i];
      for (int i = 0; i < 9; ++i) total += w_rot * dR[i] * dR[i];
      for (int j = 0; j < nj; ++j) {
        const double* Tj = T + 16 * j;
        const double a[3] = {Tj[2], Tj[6], Tj[10]}, o[3] = {Tj[3], Tj[7], Tj[11]};
        const double rel[3] = {E[3] - o[0], E[7] - o[1], E[11] - o[2]};
        const double vt[3] = {a[1] * rel[2] - a[2] * rel[1], a[2] * rel[0] - a[0] * rel[2],
                              a[0] * rel[1] - a[1] * rel[0]};
        double gj = 0.0;
        for (int i = 0; i < 3; ++i) gj += 2.0 * w_pos * dt[i] * vt[i];
        /* dR/dq_j = [a]x R: column k of R rotates as a x R_k */
        for (int k = 0; k < 3; ++k) {
          const double Rk[3] = {E[k], E[4 + k], E[8 + k]};
          const double v[3] = {a[1] * Rk[2] - a[2] * Rk[1], a[2] * Rk[0] - a[0] * Rk[2],
                               a[0] * Rk[1] - a[1] * Rk[0]};
          for (int i = 0; i < 3; ++i) gj += 2.0 * w_rot * dR[3 * i + k] * v[i];
        }
        const double qj = qc[j];
        if (qj > q_hi[j]) {
          total += w_bound * (qj - q_hi[j]) * (qj - q_hi[j]);
          gj += 2.0 * w_bound * (qj - q_hi[j]);
        } else if (qj < q_lo[j]) {
          total += w_bound * (q_lo[j] - qj) * (q_lo[j] - qj);
          gj -= 2.0 * w_bound * (q_lo[j] - qj);
        }
        grad[(int64_t)nj * c + j] += gj;
      }
      cost[c] = total;
    }
    free(T);
  }
  free(pos);
  free(ccost);
  free(dist);
  free(g);
}

void or_lbfgs_direction(int dim, int m, const double* s, const double* y, const double* g,
                        double* d) {
  double alpha[64], rho[64];
  for (int i = 0; i < dim; ++i) d[i] = -g[i];
  for (int k = m - 1; k >= 0; --k) { /* newest to oldest */
    double sy = 0.0, sq = 0.0;
    for (int i = 0; i < dim; ++i) {
      sy += s[k * dim + i] * y[k * dim + i];
      sq += s[k * dim + i] * d[i];
    }
    rho[k] = 1.0 / sy;
    alpha[k] = rho[k] * sq;
    for (int i = 0; i < dim; ++i) d[i] -= alpha[k] * y[k * dim + i];
  }
  if (m > 0) {
    double sy = 0.0, yy = 0.0;
    for (int i = 0; i < dim; ++i) {
      sy += s[(m - 1) * dim + i] * y[(m - 1) * dim + i];
      yy += y[(m - 1) * dim + i] * y[(m - 1) * dim + i];
    }
    for (int i = 0; i < dim; ++i) d[i] *= sy / yy;
  }
  for (int k = 0; k < m; ++k) { /* oldest to newest */
    double yr = 0.0;
    for (int i = 0; i < dim; ++i) yr += y[k * dim + i] * d[i];
    const double beta = rho[k] * yr;
    for (int i = 0; i < dim; ++i) d[i] += (alpha[k] - beta) * s[k * dim + i];
  }
}
