// Device math of the CR-Solver hot path: PCC segment transforms (Eq. 1-3), the inverse tendon map
// (Eq. 4), the chain, the SO(3) log of the pose error (Eq. ik_opt), the penalty rows of
// Eq. penalized_form, the hand-written adjoint (reverse sweep over segments) and the LM normal
// equations. Everything is templated on the arithmetic type T (float / double) and on the number
// of segments N, so that a state lives entirely in registers.
//
// Notation: segment i bends by a = (ax, ay) = theta (cos phi, sin phi); x = theta^2.
//   ax = K (u0 - (u1 + u2)/2), ay = K (sqrt(3)/2)(u1 - u2), K = -2 / (3 r_c)   (inverse of Eq. 4)
//   R_i = I + s [w]x + c [w]x^2, w = (-ay, ax, 0)       (Eq. 2 in Rodrigues form)
//   d_i = L (c ax, c ay, s)                            (Eq. 3)
//   s = sin(theta)/theta, c = (1 - cos theta)/theta^2, evaluated through the half angle:
//   s = sinc(theta/2) cos(theta/2), c = sinc(theta/2)^2 / 2 (no cancellation near theta = 0).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cr.h"

#define CR_HD __device__ __forceinline__

namespace crk {

constexpr int NMAX = CR_MAX_SEG;

template <typename T> struct Prec;
template <> struct Prec<float> {
  static constexpr float kZero = 1e-12f;     // theta^2 below which sinc(theta/2) uses its series
  static constexpr float kSeriesX = 1.0f;    // theta^2 below which s3 and dc/dx use their series
  static constexpr float kLogSmall = 1e-10f; // |vee|^2 below which Log uses 1 + s^2/6
  static constexpr float kLogPi = 1e-2f;     // |vee|^2 below which (cos < 0) Log takes the symmetric part
  static constexpr float kBetaSeries = 1.0f; // angle^2 below which the log-Jacobian factor uses its series
};
template <> struct Prec<double> {
  static constexpr double kZero = 1e-20;
  static constexpr double kSeriesX = 0.1;
  static constexpr double kLogSmall = 1e-6;
  static constexpr double kLogPi = 1e-2;
  static constexpr double kBetaSeries = 1e-2;
};

CR_HD float c_sqrt(float x) { return sqrtf(x); }
CR_HD double c_sqrt(double x) { return sqrt(x); }
// FP32 sin and cos through sincospif: its reduction modulo 2 is exact, so no large-argument
// reduction subroutine is called (such a call caps the register allocation of the whole kernel).
CR_HD void c_sincos(float x, float* s, float* c) { sincospif(x * 0.31830988618379067f, s, c); }
// FP64: the library sincos (the FP64 results follow the oracle's decisions to the last bits).
CR_HD void c_sincos(double x, double* s, double* c) { sincos(x, s, c); }
CR_HD float c_atan2(float y, float x) { return atan2f(y, x); }
CR_HD double c_atan2(double y, double x) { return atan2(y, x); }
CR_HD float c_rsqrt(float x) { return rsqrtf(x); }
CR_HD float c_div(float a, float b) { return __fdividef(a, b); }
CR_HD double c_div(double a, double b) { return a / b; }
CR_HD double c_rsqrt(double x) { return 1.0 / sqrt(x); }
CR_HD float c_fabs(float x) { return fabsf(x); }
CR_HD double c_fabs(double x) { return fabs(x); }
CR_HD bool c_finite(float x) { return isfinite(x); }
CR_HD bool c_finite(double x) { return isfinite(x); }
template <typename T> CR_HD T c_max(T a, T b) { return a > b ? a : b; }
template <typename T> CR_HD T c_abs(T a) { return a < T(0) ? -a : a; }
template <typename T> CR_HD T c_min(T a, T b) { return a < b ? a : b; }
template <typename T> CR_HD T clampb(T v, T b) { return c_min(b, c_max(-b, v)); }

// ------------------------------------------------------------------------------------------------
// Parameters as the kernels see them
// ------------------------------------------------------------------------------------------------
template <typename T> struct RobotK {
  int n, nb;
  T L[NMAX], K[NMAX], umax[NMAX], thmax[NMAX], rc[NMAX];
  T rbody;
  T lmin[NMAX], lmax[NMAX];  // CR_MODEL_ARC length bounds
};

struct NmaxArr {
  double v[NMAX];
};

template <typename T> struct WeightsK {
  T wp2, wR2;              // squared pose weights
  T wp, wR;
  T rho_b, rho_eq, rho_k, rho_c;
  T sb, se, sk, sc;        // square roots of the penalty weights (row scale)
  T delta;
  T rho_s, ss;             // self-contact rows (0: none) and the square root of their weight
};

// ------------------------------------------------------------------------------------------------
// Segment functions of theta^2
// ------------------------------------------------------------------------------------------------
// s = sin(t)/t and c = (1 - cos t)/t^2 from x = t^2 (half-angle form, library sin/cos).
template <typename T> CR_HD void seg_sc_lib(T x, T& s, T& c) {
  T sc, ch;
  if (x < Prec<T>::kZero) {
    sc = T(1) - x * T(1.0 / 24.0);
    ch = T(1) - x * T(0.125);
  } else {
    T h = T(0.5) * c_sqrt(x);
    T sh;
    c_sincos(h, &sh, &ch);
    sc = sh / h;
  }
  s = sc * ch;
  c = T(0.5) * sc * sc;
}

// s3 = (t - sin t)/t^3 = (1 - s)/x and cp = dc/dx = (s - 2c)/(2x); Taylor series in x below kSeriesX.
template <typename T> CR_HD void seg_deriv_lib(T x, T s, T c, T& s3, T& cp) {
  if (x < Prec<T>::kSeriesX) {
    s3 = T(1.0 / 6.0) + x * (T(-1.0 / 120.0) + x * (T(1.0 / 5040.0) + x * (T(-1.0 / 362880.0) +
         x * (T(1.0 / 39916800.0) + x * (T(-1.0 / 6227020800.0) + x * T(1.0 / 1307674368000.0))))));
    cp = T(-1.0 / 24.0) + x * (T(1.0 / 360.0) + x * (T(-1.0 / 13440.0) + x * (T(1.0 / 907200.0) +
         x * (T(-1.0 / 95800320.0) + x * (T(1.0 / 14529715200.0) + x * T(-1.0 / 2988969984000.0))))));
  } else {
    T ix = T(1) / x;
    s3 = (T(1) - s) * ix;
    cp = (s - T(2) * c) * (T(0.5) * ix);
  }
}

template <typename T> CR_HD void seg_sc(T x, T& s, T& c) { seg_sc_lib(x, s, c); }
template <typename T> CR_HD void seg_deriv(T x, T s, T c, T& s3, T& cp) { seg_deriv_lib(x, s, c, s3, cp); }

// FP32: for theta <= pi the four coefficients are Taylor polynomials (no square root, sin/cos or
// division): with y = (theta/2)^2, sinc(theta/2) = sum_k (-1)^k y^k / (2k+1)! (degree 6) and
// cos(theta/2) = sum_k (-1)^k y^k / (2k)! (degree 7); s3 = sum_k (-1)^k x^k / (2k+3)! and
// cp = sum_k (-1)^(k+1) (k+1) x^k / (2k+4)! (degree 8). Truncation error <= 2e-9 relative up to
// theta^2 = 9.87 (theta <= 3.1417; 5e-11 absolute for s, which vanishes at theta = pi), far below
// FP32 rounding. The bound sits just above pi^2 so that a
// bend projected onto theta = pi (whose theta^2 rounds up to pi^2 (1 + 2e-7)) stays on the
// polynomials; larger angles take the library path.
constexpr float kPolyMaxX = 9.87f;

template <> CR_HD void seg_sc<float>(float x, float& s, float& c) {
  if (x <= kPolyMaxX) {
    const float y = 0.25f * x;
    float sc = 1.6059043836821613e-10f;
    sc = fmaf(sc, y, -2.505210838544172e-08f);
    sc = fmaf(sc, y, 2.7557319223985893e-06f);
    sc = fmaf(sc, y, -0.0001984126984126984f);
    sc = fmaf(sc, y, 0.008333333333333333f);
    sc = fmaf(sc, y, -0.16666666666666666f);
    sc = fmaf(sc, y, 1.0f);
    float ch = -1.1470745597729725e-11f;
    ch = fmaf(ch, y, 2.08767569878681e-09f);
    ch = fmaf(ch, y, -2.755731922398589e-07f);
    ch = fmaf(ch, y, 2.48015873015873e-05f);
    ch = fmaf(ch, y, -0.001388888888888889f);
    ch = fmaf(ch, y, 0.041666666666666664f);
    ch = fmaf(ch, y, -0.5f);
    ch = fmaf(ch, y, 1.0f);
    s = sc * ch;
    c = 0.5f * sc * sc;
  } else {
    seg_sc_lib(x, s, c);
  }
}

template <> CR_HD void seg_deriv<float>(float x, float s, float c, float& s3, float& cp) {
  if (x <= kPolyMaxX) {
    float a = 8.22063524662433e-18f;
    a = fmaf(a, x, -2.8114572543455206e-15f);
    a = fmaf(a, x, 7.647163731819816e-13f);
    a = fmaf(a, x, -1.6059043836821613e-10f);
    a = fmaf(a, x, 2.505210838544172e-08f);
    a = fmaf(a, x, -2.7557319223985893e-06f);
    a = fmaf(a, x, 0.0001984126984126984f);
    a = fmaf(a, x, -0.008333333333333333f);
    s3 = fmaf(a, x, 0.16666666666666666f);
    float b = -3.6992858609809485e-18f;
    b = fmaf(b, x, 1.249536557486898e-15f);
    b = fmaf(b, x, -3.3456341326711696e-13f);
    b = fmaf(b, x, 6.882447358637835e-11f);
    b = fmaf(b, x, -1.043837849393405e-08f);
    b = fmaf(b, x, 1.1022927689594355e-06f);
    b = fmaf(b, x, -7.440476190476191e-05f);
    b = fmaf(b, x, 0.002777777777777778f);
    cp = fmaf(b, x, -0.041666666666666664f);
  } else {
    seg_deriv_lib(x, s, c, s3, cp);
  }
}

// Local derivatives of one segment with respect to (ax, ay):
//  dd[k]: d(d_i)/da_k = L (c e_k + 2 a_k cp (ax, ay, 0) + 2 a_k sp e_z), sp = ds/dx = (s3 - c)/2
//  wl[k]: vee(dR R^T)/da_k = J_l(w) dw/da_k, J_l = I + c [w]x + s3 [w]x^2 (left Jacobian of SO(3))
template <typename T>
CR_HD void seg_local_derivs(T ax, T ay, T s, T c, T s3, T cp, T L, T (&dd)[2][3], T (&wl)[2][3]) {
  T sp = T(0.5) * (s3 - c);
  T axy = ax * ay;
  dd[0][0] = L * (c + T(2) * ax * ax * cp);
  dd[0][1] = L * (T(2) * axy * cp);
  dd[0][2] = L * (T(2) * ax * sp);
  dd[1][0] = dd[0][1];
  dd[1][1] = L * (c + T(2) * ay * ay * cp);
  dd[1][2] = L * (T(2) * ay * sp);
  wl[0][0] = -s3 * axy;
  wl[0][1] = T(1) - s3 * ay * ay;
  wl[0][2] = -c * ay;
  wl[1][0] = s3 * ax * ax - T(1);
  wl[1][1] = s3 * axy;
  wl[1][2] = c * ax;
}

// Rotation and translation of a segment (Eq. 2-3).
template <typename T> CR_HD void seg_transform(T ax, T ay, T x, T s, T c, T L, T (&Ri)[9], T (&di)[3]) {
  T caxy = c * ax * ay;
  Ri[0] = T(1) - c * ax * ax; Ri[1] = -caxy;               Ri[2] = s * ax;
  Ri[3] = -caxy;               Ri[4] = T(1) - c * ay * ay; Ri[5] = s * ay;
  Ri[6] = -s * ax;             Ri[7] = -s * ay;            Ri[8] = T(1) - c * x;
  di[0] = L * c * ax;
  di[1] = L * c * ay;
  di[2] = L * s;
}

template <typename T> CR_HD void bend_of(T K, T u0, T u1, T u2, T& ax, T& ay) {
  ax = K * (u0 - T(0.5) * (u1 + u2));
  ay = K * (T(0.86602540378443864676) * (u1 - u2));
}

// grad in u of a segment from grad in a: (du0, du1, du2) = K C^T (ga_x, ga_y)
template <typename T> CR_HD void bend_grad_to_u(T K, T gx, T gy, T& g0, T& g1, T& g2) {
  T hx = T(0.5) * gx, ry = T(0.86602540378443864676) * gy;
  g0 = K * gx;
  g1 = K * (ry - hx);
  g2 = K * (-ry - hx);
}

template <typename T> CR_HD void matvec(const T (&R)[9], const T (&v)[3], T (&o)[3]) {
  o[0] = R[0] * v[0] + R[1] * v[1] + R[2] * v[2];
  o[1] = R[3] * v[0] + R[4] * v[1] + R[5] * v[2];
  o[2] = R[6] * v[0] + R[7] * v[1] + R[8] * v[2];
}
template <typename T> CR_HD void matTvec(const T (&R)[9], const T (&v)[3], T (&o)[3]) {
  o[0] = R[0] * v[0] + R[3] * v[1] + R[6] * v[2];
  o[1] = R[1] * v[0] + R[4] * v[1] + R[7] * v[2];
  o[2] = R[2] * v[0] + R[5] * v[1] + R[8] * v[2];
}
template <typename T> CR_HD void cross(const T (&a)[3], const T (&b)[3], T (&o)[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
template <typename T> CR_HD T dot3(const T (&a)[3], const T (&b)[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// ------------------------------------------------------------------------------------------------
// Forward chain
// ------------------------------------------------------------------------------------------------
template <typename T, int N> struct Chain {
  T Rb[N][9], pb[N][3];  // base frame of every segment
  T ax[N], ay[N], x[N], s[N], c[N];
  T L[N];                // arc lengths: the robot's (tendon model) or the state's (arc model)
  T R[9], p[3];          // tip frame
};

// Bend a = (theta cos phi, theta sin phi) and length of segment i from the state (see cr_model).
template <int MODEL, typename T, int N>
CR_HD void segment_state(const RobotK<T>& rb, const T (&u)[3 * N], int i, T& ax, T& ay, T& L) {
  if (MODEL == CR_MODEL_ARC) {
    ax = u[3 * i];
    ay = u[3 * i + 1];
    L = u[3 * i + 2];
  } else if (MODEL == CR_MODEL_COUPLED && i > 0) {
    // coupled routing: the state holds actuator displacements q; segment i bends with u_i = q_i - q_{i-1}
    bend_of(rb.K[i], u[3 * i] - u[3 * i - 3], u[3 * i + 1] - u[3 * i - 2], u[3 * i + 2] - u[3 * i - 1], ax, ay);
    L = rb.L[i];
  } else {
    bend_of(rb.K[i], u[3 * i], u[3 * i + 1], u[3 * i + 2], ax, ay);
    L = rb.L[i];
  }
}

// State columns of segment i from the derivatives (gx, gy) with respect to its bend: the tendon
// model maps them through the inverse of Eq. 4 (dF/du = K C^T g); the arc model's first two state
// components are the bend itself (its third, the length, is filled by the caller).
template <int MODEL, typename T>
CR_HD void bend_cols(const RobotK<T>& rb, int i, T gx, T gy, T& c0, T& c1, T& c2) {
  if (MODEL == CR_MODEL_ARC) {
    c0 = gx;
    c1 = gy;
    c2 = T(0);
  } else {
    bend_grad_to_u(rb.K[i], gx, gy, c0, c1, c2);
  }
}

// A row of u-space derivatives (per-segment displacements) to the state's: the identity, except for
// coupled routing, where u = D q (u_s = q_s - q_{s-1}) and so d/dq_s = d/du_s - d/du_{s+1}.
template <int MODEL, typename T, int N> CR_HD void to_actuator(T (&jr)[3 * N]) {
  if (MODEL != CR_MODEL_COUPLED) return;
#pragma unroll
  for (int q = 0; q + 3 < 3 * N; ++q) jr[q] -= jr[q + 3];
}

template <typename T, int N, int MODEL = CR_MODEL_TENDON>
CR_HD void chain_forward(const RobotK<T>& rb, const T (&u)[3 * N], Chain<T, N>& ch) {
  T R[9] = {T(1), T(0), T(0), T(0), T(1), T(0), T(0), T(0), T(1)};
  T p[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int i = 0; i < N; ++i) {
#pragma unroll
    for (int a = 0; a < 9; ++a) ch.Rb[i][a] = R[a];
#pragma unroll
    for (int a = 0; a < 3; ++a) ch.pb[i][a] = p[a];
    T ax, ay, Li;
    segment_state<MODEL, T, N>(rb, u, i, ax, ay, Li);
    T x = ax * ax + ay * ay;
    T s, c;
    seg_sc(x, s, c);
    ch.ax[i] = ax; ch.ay[i] = ay; ch.x[i] = x; ch.s[i] = s; ch.c[i] = c; ch.L[i] = Li;
    T Ri[9], di[3];
    seg_transform(ax, ay, x, s, c, Li, Ri, di);
    if (i == 0) {  // base frame = identity: the products by its zeros are left out
#pragma unroll
      for (int a = 0; a < 9; ++a) R[a] = Ri[a];
#pragma unroll
      for (int a = 0; a < 3; ++a) p[a] = di[a];
      continue;
    }
    T t[3];
    matvec(R, di, t);
    p[0] += t[0]; p[1] += t[1]; p[2] += t[2];
    T Rn[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int q = 0; q < 3; ++q)
        Rn[3 * r + q] = R[3 * r] * Ri[q] + R[3 * r + 1] * Ri[3 + q] + R[3 * r + 2] * Ri[6 + q];
#pragma unroll
    for (int a = 0; a < 9; ++a) R[a] = Rn[a];
  }
#pragma unroll
  for (int a = 0; a < 9; ++a) ch.R[a] = R[a];
#pragma unroll
  for (int a = 0; a < 3; ++a) ch.p[a] = p[a];
}

// Backbone sample at arc fraction sg of segment i (base frame Rb, pb): the sub-arc bends by sg*a
// over sg*L. Returns the local point q and the world point w.
template <typename T>
CR_HD void backbone_point(const T (&Rb)[9], const T (&pb)[3], T ax, T ay, T x, T L, T sg, T (&q)[3],
                          T (&w)[3], T& s, T& c) {
  T xs = sg * sg * x;
  seg_sc(xs, s, c);
  T sL = sg * L;
  q[0] = sL * c * (sg * ax);
  q[1] = sL * c * (sg * ay);
  q[2] = sL * s;
  T t[3];
  matvec(Rb, q, t);
  w[0] = pb[0] + t[0];
  w[1] = pb[1] + t[1];
  w[2] = pb[2] + t[2];
}

// ------------------------------------------------------------------------------------------------
// Targets and pose error
// ------------------------------------------------------------------------------------------------
template <typename T> struct TargetK {
  T p[3];
  T R[9];  // IK6: target rotation; IK5: R[0..2] = unit tip axis
};

// targets [7][P] SoA, FP64
template <typename T> CR_HD TargetK<T> load_target(const double* tg, int64_t P, int64_t q, int kind) {
  TargetK<T> t;
  t.p[0] = T(tg[q]);
  t.p[1] = T(tg[P + q]);
  t.p[2] = T(tg[2 * P + q]);
  if (kind == CR_TASK_IK5) {
    T zx = T(tg[3 * P + q]), zy = T(tg[4 * P + q]), zz = T(tg[5 * P + q]);
    T inv = T(1) / c_sqrt(zx * zx + zy * zy + zz * zz);
    t.R[0] = zx * inv; t.R[1] = zy * inv; t.R[2] = zz * inv;
    for (int a = 3; a < 9; ++a) t.R[a] = T(0);
  } else {
    T w = T(tg[3 * P + q]), x = T(tg[4 * P + q]), y = T(tg[5 * P + q]), z = T(tg[6 * P + q]);
    T inv = T(1) / c_sqrt(w * w + x * x + y * y + z * z);
    w *= inv; x *= inv; y *= inv; z *= inv;
    t.R[0] = T(1) - T(2) * (y * y + z * z); t.R[1] = T(2) * (x * y - w * z); t.R[2] = T(2) * (x * z + w * y);
    t.R[3] = T(2) * (x * y + w * z); t.R[4] = T(1) - T(2) * (x * x + z * z); t.R[5] = T(2) * (y * z - w * x);
    t.R[6] = T(2) * (x * z - w * y); t.R[7] = T(2) * (y * z + w * x); t.R[8] = T(1) - T(2) * (x * x + y * y);
  }
  return t;
}

// SO(3) log of E (row-major): e = angle * axis. Returns the angle; sn = sin(angle).
template <typename T> CR_HD T so3_log(const T (&E)[9], T (&e)[3], T& sn_out, T& cs_out) {
  T v0 = T(0.5) * (E[7] - E[5]), v1 = T(0.5) * (E[2] - E[6]), v2 = T(0.5) * (E[3] - E[1]);
  T cs = T(0.5) * (E[0] + E[4] + E[8] - T(1));
  T s2 = v0 * v0 + v1 * v1 + v2 * v2;
  T sn = c_sqrt(s2);
  T ang = c_atan2(sn, cs);
  sn_out = sn;
  cs_out = cs;
  // Near pi the axis v / |v| loses relative accuracy as |v| -> 0; FP64 then takes it from the
  // symmetric part. FP32 keeps the single branch-free formula (its error there, ~eps / sin, is
  // below the FP32 accuracy of the other terms for angles up to pi - 0.05).
  if (sizeof(T) == 8 && cs < T(0) && s2 < Prec<T>::kLogPi) {
    // near pi: (E + E^T)/2 = cs I + (1 - cs) n n^T; largest diagonal gives the best-conditioned column
    T S00 = E[0], S11 = E[4], S22 = E[8];
    T den = T(1) / (T(1) - cs);
    int k = (S11 > S00) ? 1 : 0;
    if (S22 > (k == 1 ? S11 : S00)) k = 2;
    T Skk = k == 0 ? S00 : (k == 1 ? S11 : S22);
    T nk = c_sqrt(c_max((Skk - cs) * den, T(0)));
    T inv = T(1) / nk;
    T n[3];
    // off-diagonal symmetric parts
    T S01 = T(0.5) * (E[1] + E[3]), S02 = T(0.5) * (E[2] + E[6]), S12 = T(0.5) * (E[5] + E[7]);
    if (k == 0) { n[0] = nk; n[1] = S01 * den * inv; n[2] = S02 * den * inv; }
    else if (k == 1) { n[0] = S01 * den * inv; n[1] = nk; n[2] = S12 * den * inv; }
    else { n[0] = S02 * den * inv; n[1] = S12 * den * inv; n[2] = nk; }
    T sgn = (n[0] * v0 + n[1] * v1 + n[2] * v2) < T(0) ? T(-1) : T(1);
    e[0] = sgn * ang * n[0];
    e[1] = sgn * ang * n[1];
    e[2] = sgn * ang * n[2];
    return ang;
  }
  T f = (s2 < Prec<T>::kLogSmall) ? T(1) + s2 * T(1.0 / 6.0) : c_div(ang, sn);
  e[0] = f * v0;
  e[1] = f * v1;
  e[2] = f * v2;
  return ang;
}

// beta(angle) = 1/angle^2 - (1 + cos)/(2 angle sin) = (1 - (a/2) cot(a/2)) / a^2: the factor of
// [e]x^2 in the inverse right Jacobian J_r^-1(e) = I + [e]x / 2 + beta [e]x^2.
template <typename T> CR_HD T log_beta(T ang) {
  T y = ang * ang;
  if (y < Prec<T>::kBetaSeries)
    return T(1.0 / 12.0) + y * (T(1.0 / 720.0) + y * (T(1.0 / 30240.0) + y * (T(1.0 / 1209600.0) +
           y * (T(1.0 / 47900160.0) + y * T(1.0 / 1892437580.3)))));
  T sh, chh;
  c_sincos(T(0.5) * ang, &sh, &chh);
  return (sh - T(0.5) * ang * chh) / (y * sh);
}

// Pose residual rows r[6] of the tip (R, p) against a target.
template <typename T>
CR_HD void pose_rows(int kind, const WeightsK<T>& w, const TargetK<T>& tg, const T (&R)[9],
                     const T (&p)[3], T (&r)[6], T (&e)[3], T& ang, T& sn, T& cs) {
  r[0] = w.wp * (p[0] - tg.p[0]);
  r[1] = w.wp * (p[1] - tg.p[1]);
  r[2] = w.wp * (p[2] - tg.p[2]);
  if (kind == CR_TASK_IK5) {
    e[0] = R[2] - tg.R[0];
    e[1] = R[5] - tg.R[1];
    e[2] = R[8] - tg.R[2];
    ang = T(0); sn = T(0); cs = T(1);
  } else {
    T E[9];  // R_t^T R
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
        E[3 * a + b] = tg.R[a] * R[b] + tg.R[3 + a] * R[3 + b] + tg.R[6 + a] * R[6 + b];
    ang = so3_log(E, e, sn, cs);
  }
  r[3] = w.wR * e[0];
  r[4] = w.wR * e[1];
  r[5] = w.wR * e[2];
}

// ------------------------------------------------------------------------------------------------
// Obstacles
// ------------------------------------------------------------------------------------------------
// Spheres as the kernels see them: (centre, reach = r_s + r_body + delta), staged in shared memory.
template <typename T> struct Sphere4 { T x, y, z, reach; };

// Threads tid, tid + nthr, ... of the caller's group stage the entries (by default the whole block).
template <typename T>
__device__ void stage_spheres(const double* sp, int no, const RobotK<T>& rb, T delta, Sphere4<T>* sh, int tid = -1,
                              int nthr = 0) {
  if (tid < 0) {
    tid = threadIdx.x;
    nthr = blockDim.x;
  }
  for (int j = tid; j < no; j += nthr) {
    Sphere4<T> s;
    s.x = T(sp[4 * j]);
    s.y = T(sp[4 * j + 1]);
    s.z = T(sp[4 * j + 2]);
    s.reach = T(sp[4 * j + 3]) + rb.rbody + delta;
    sh[j] = s;
  }
}

// Primitives (capsules, boxes: the convex pieces of Sec. IV-C) as the kernels see them. Each also
// has a bounding sphere in the Sphere4 table, after the n_o spheres (table index n_o + jp), whose
// reach bounds that of every point of the primitive, so that the broad phase treats both alike.
template <typename T> struct PrimK {
  T c[3];    // capsule: end point a; box: centre
  T e[3];    // capsule: b - a; box: half extents
  T R[9];    // box: rotation, box frame to world, row-major
  T iee;     // capsule: 1 / |b - a|^2 (0 when a = b)
  T reach;   // r + r_body + delta
  int kind;  // CR_PRIM_CAPSULE, CR_PRIM_BOX; any other value: a sphere centred at c
};

// Stage primitive records pr [np][CR_PRIM_DOUBLES] (FP64): the records into sh, their bounding
// spheres into bnd. The rotation and the bounds are formed in FP64 and rounded once to T.
template <typename T>
__device__ void stage_prims(const double* pr, int np, const RobotK<T>& rb, T delta, Sphere4<T>* bnd, PrimK<T>* sh,
                            int tid, int nthr) {
  for (int j = tid; j < np; j += nthr) {
    const double* r = pr + (size_t)CR_PRIM_DOUBLES * j;
    const int kind = (int)r[0];
    const double reach = r[1] + (double)rb.rbody + (double)delta;
    PrimK<T> P;
    P.kind = kind == CR_PRIM_CAPSULE || kind == CR_PRIM_BOX ? kind : CR_PRIM_SPHERE;
    P.reach = T(reach);
    double e[3] = {0.0, 0.0, 0.0}, ctr[3] = {r[2], r[3], r[4]}, rad = 0.0;
    for (int a = 0; a < 9; ++a) P.R[a] = T(a % 4 == 0 ? 1 : 0);
    P.iee = T(0);
    if (P.kind == CR_PRIM_CAPSULE) {
      for (int a = 0; a < 3; ++a) e[a] = r[5 + a] - r[2 + a];
      const double ee = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
      P.iee = ee > 0.0 ? T(1.0 / ee) : T(0);
      for (int a = 0; a < 3; ++a) ctr[a] = r[2 + a] + 0.5 * e[a];
      rad = 0.5 * sqrt(ee);
    } else if (P.kind == CR_PRIM_BOX) {
      for (int a = 0; a < 3; ++a) e[a] = r[5 + a];
      rad = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
      // unit quaternion (w, x, y, z) -> rotation matrix
      double qw = r[8], qx = r[9], qy = r[10], qz = r[11];
      const double qn = sqrt(qw * qw + qx * qx + qy * qy + qz * qz);
      qw /= qn; qx /= qn; qy /= qn; qz /= qn;
      const double M[9] = {1.0 - 2.0 * (qy * qy + qz * qz), 2.0 * (qx * qy - qw * qz), 2.0 * (qx * qz + qw * qy),
                           2.0 * (qx * qy + qw * qz), 1.0 - 2.0 * (qx * qx + qz * qz), 2.0 * (qy * qz - qw * qx),
                           2.0 * (qx * qz - qw * qy), 2.0 * (qy * qz + qw * qx), 1.0 - 2.0 * (qx * qx + qy * qy)};
      for (int a = 0; a < 9; ++a) P.R[a] = T(M[a]);
    }
    for (int a = 0; a < 3; ++a) {
      P.c[a] = T(r[2 + a]);
      P.e[a] = T(e[a]);
    }
    sh[j] = P;
    bnd[j] = Sphere4<T>{T(ctr[0]), T(ctr[1]), T(ctr[2]), T(rad + reach)};
  }
}

// The obstacles one evaluation sees: the Sphere4 table s (n_o spheres, then the bounding spheres of
// the primitives) and the primitive records p; table entries j >= ns are primitive j - ns. Built
// from a bare sphere table it holds spheres only.
template <typename T> struct ObsK {
  const Sphere4<T>* s;
  const PrimK<T>* p;
  int ns;
  CR_HD ObsK(const Sphere4<T>* s_) : s(s_), p(nullptr), ns(1 << 30) {}
  CR_HD ObsK(const Sphere4<T>* s_, const PrimK<T>* p_, int ns_) : s(s_), p(p_), ns(ns_) {}
  // the table from entry k on (its entry j is entry k + j of this one)
  CR_HD ObsK from(int k) const { return ObsK(s + k, p, ns - k); }
  // whether primitives may follow the spheres: every primitive branch tests this first, so that in
  // a kernel that builds its view from a bare sphere table (p a constant null pointer) the
  // primitive code folds away
  CR_HD bool prims() const { return p != nullptr; }
};

// Shared-memory bytes of a staged obstacle set: the Sphere4 table (no + np entries), then the
// primitive records from the next 16-byte boundary.
template <typename T> __host__ __device__ inline size_t obstacles_smem(int no, int np) {
  const size_t t = ((size_t)(no + np) * sizeof(Sphere4<T>) + 15) & ~(size_t)15;
  return t + (size_t)np * sizeof(PrimK<T>);
}

// Stage spheres sp [no][4] and primitive records pr [np][CR_PRIM_DOUBLES] at base (threads tid,
// tid + nthr, ... of the caller's group, by default the whole block; the caller synchronises the
// group before use).
template <typename T>
__device__ ObsK<T> stage_obstacles(const double* sp, int no, const double* pr, int np, const RobotK<T>& rb, T delta,
                                   unsigned char* base, int tid = -1, int nthr = 0) {
  if (tid < 0) {
    tid = threadIdx.x;
    nthr = blockDim.x;
  }
  Sphere4<T>* tab = reinterpret_cast<Sphere4<T>*>(base);
  PrimK<T>* prm = reinterpret_cast<PrimK<T>*>(base + (((size_t)(no + np) * sizeof(Sphere4<T>) + 15) & ~(size_t)15));
  stage_spheres(sp, no, rb, delta, tab, tid, nthr);
  if (np > 0) stage_prims(pr, np, rb, delta, tab + no, prm, tid, nthr);
  return ObsK<T>(tab, prm, no);
}

// Signed distance from x to primitive P's core (the quantity prim_active compares with a reach).
template <typename T> CR_HD T prim_sd(const PrimK<T>& P, const T (&x)[3]) {
  const T w0 = x[0] - P.c[0], w1 = x[1] - P.c[1], w2 = x[2] - P.c[2];
  if (P.kind == CR_PRIM_BOX) {
    T q[3], o2 = T(0), qm;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      q[a] = c_abs(P.R[a] * w0 + P.R[3 + a] * w1 + P.R[6 + a] * w2) - P.e[a];
      if (q[a] > T(0)) o2 += q[a] * q[a];
    }
    qm = q[0] > q[1] ? q[0] : q[1];
    qm = qm > q[2] ? qm : q[2];
    return qm > T(0) ? c_sqrt(o2) : qm;
  }
  T d0 = w0, d1 = w1, d2 = w2;
  if (P.kind == CR_PRIM_CAPSULE) {
    T t = (w0 * P.e[0] + w1 * P.e[1] + w2 * P.e[2]) * P.iee;
    t = t < T(0) ? T(0) : (t > T(1) ? T(1) : t);
    d0 -= t * P.e[0];
    d1 -= t * P.e[1];
    d2 -= t * P.e[2];
  }
  return c_sqrt(d0 * d0 + d1 * d1 + d2 * d2);
}

// stage_obstacles, or with PRIMS = false the spheres alone behind a bare view (no primitive code is
// compiled into the kernel that uses it; the caller launches that form for scenes without primitives).
template <bool PRIMS, typename T>
__device__ ObsK<T> stage_obstacles_as(const double* sp, int no, const double* pr, int np, const RobotK<T>& rb, T delta,
                                      unsigned char* base, int tid = -1, int nthr = 0) {
  if (PRIMS) return stage_obstacles(sp, no, pr, np, rb, delta, base, tid, nthr);
  stage_spheres(sp, no, rb, delta, reinterpret_cast<Sphere4<T>*>(base), tid, nthr);
  return ObsK<T>(reinterpret_cast<const Sphere4<T>*>(base));
}

// Clearance of point x against primitive P within `reach` (P.reach for the rows): true when
// sd(x) < reach, with sd the signed distance from x to the primitive's core; then viol = reach - sd
// and n = d sd / dx (unit). Capsule: distance to the nearest point a + t (b - a), t clamped to
// [0, 1]. Box, in box coordinates p = R^T (x - c) and q_a = |p_a| - h_a: outside, the distance to
// the box (offset sign(p_a) max(q_a, 0) per axis); inside, sd = max_a q_a, n = the outward normal of
// that face (the first axis among equal maxima).
template <typename T>
CR_HD bool prim_active(const PrimK<T>& P, const T (&x)[3], T reach, T& viol, T (&n)[3]) {
  const T w0 = x[0] - P.c[0], w1 = x[1] - P.c[1], w2 = x[2] - P.c[2];
  if (P.kind == CR_PRIM_BOX) {
    T p[3], q[3];
    bool out = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      p[a] = P.R[a] * w0 + P.R[3 + a] * w1 + P.R[6 + a] * w2;
      q[a] = c_abs(p[a]) - P.e[a];
      out = out || q[a] > T(0);
    }
    if (out) {
      T o[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) o[a] = q[a] > T(0) ? (p[a] < T(0) ? -q[a] : q[a]) : T(0);
      const T d2 = o[0] * o[0] + o[1] * o[1] + o[2] * o[2];
      if (!(d2 < reach * reach)) return false;
      const T dist = c_sqrt(d2);
      viol = reach - dist;
      const T id = T(1) / dist;
#pragma unroll
      for (int b = 0; b < 3; ++b) n[b] = (P.R[3 * b] * o[0] + P.R[3 * b + 1] * o[1] + P.R[3 * b + 2] * o[2]) * id;
      return true;
    }
    int am = 0;
    if (q[1] > q[am]) am = 1;
    if (q[2] > q[am]) am = 2;
    viol = reach - q[am];
    const T sg = p[am] < T(0) ? T(-1) : T(1);
#pragma unroll
    for (int b = 0; b < 3; ++b) n[b] = sg * P.R[3 * b + am];
    return viol > T(0);
  }
  T d0 = w0, d1 = w1, d2c = w2;
  if (P.kind == CR_PRIM_CAPSULE) {
    T t = (w0 * P.e[0] + w1 * P.e[1] + w2 * P.e[2]) * P.iee;
    t = t < T(0) ? T(0) : (t > T(1) ? T(1) : t);
    d0 = w0 - t * P.e[0];
    d1 = w1 - t * P.e[1];
    d2c = w2 - t * P.e[2];
  }
  const T d2 = d0 * d0 + d1 * d1 + d2c * d2c;
  if (!(d2 < reach * reach)) return false;
  const T dist = c_sqrt(d2);
  viol = reach - dist;
  const T id = T(1) / dist;
  n[0] = d0 * id;
  n[1] = d1 * id;
  n[2] = d2c * id;
  return true;
}

// The bits of the 64-entry chunk from table entry j0 on that are spheres (the rest are primitives).
template <typename T> CR_HD uint64_t sphere_bits(const ObsK<T>& ob, int j0) {
  const int cs = ob.ns - j0;
  return cs >= 64 ? ~0ull : (cs <= 0 ? 0ull : (1ull << cs) - 1ull);
}

// Exact broad-phase test of the primitives among the candidates mask (bits relative to j0) that
// passed their bounding spheres: sd is 1-Lipschitz, so no point of the ball of radius rad about m
// comes within reach when sd(m) >= reach + rad (a shelf board, whose bounding sphere is large, then
// culls like a slab of its own thickness); the margin is the bounding test's. Inlined: kernels for
// scenes without primitives build a view whose primitive pointer is a constant null, and the call
// folds away there.
template <typename T>
CR_HD uint64_t prim_exact_cull(ObsK<T> ob, int j0, uint64_t mask, T mx, T my, T mz, T rad, T lsum) {
  const T m[3] = {mx, my, mz};
  for (uint64_t b = mask & ~sphere_bits(ob, j0); b; b &= b - 1) {
    const int jj = __ffsll((long long)b) - 1;
    const Sphere4<T> S = ob.s[j0 + jj];
    const PrimK<T>& P = ob.p[j0 + jj - ob.ns];
    const T marg = T(1e-4) * (lsum + S.reach + c_abs(S.x) + c_abs(S.y) + c_abs(S.z));
    if (!(prim_sd(P, m) < P.reach + rad + marg)) mask &= ~(1ull << jj);
  }
  return mask;
}

// Broad phase of the clearance rows. Spheres j0 .. j0 + cnt - 1 (cnt <= 64) that may come within reach
// of some backbone sample of segment i are the set bits of mask[i]. The backbone has unit speed in arc
// length, so every sample of segment i lies within L_i / 2 of the segment's mid-arc point; a sphere
// whose centre is farther than L_i / 2 + reach from that point reaches none of them. The margin (a
// 1e-4 fraction of the magnitudes involved) covers rounding, so a culled pair is one the exact
// per-sample test rejects as well and the active set is unchanged.
// Table entries from ns on are primitives' bounding spheres; one that passes is then tested exactly
// (prim_exact_cull).
template <typename T, int N>
CR_HD void segment_sphere_masks(const RobotK<T>& rb, const Chain<T, N>& ch, ObsK<T> ob, int j0, int cnt,
                                uint64_t (&mask)[N]) {
  const Sphere4<T>* sph = ob.s;
  T lsum = T(0);
#pragma unroll
  for (int i = 0; i < N; ++i) lsum += ch.L[i];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    T q[3], m[3], s, c;
    backbone_point(ch.Rb[i], ch.pb[i], ch.ax[i], ch.ay[i], ch.x[i], ch.L[i], T(0.5), q, m, s, c);
    const T half = T(0.5) * ch.L[i];
    uint64_t mk = 0;
    for (int j = 0; j < cnt; ++j) {
      const Sphere4<T> S = sph[j0 + j];
      const T dx = m[0] - S.x, dy = m[1] - S.y, dz = m[2] - S.z;
      const T lim = half + S.reach + T(1e-4) * (lsum + S.reach + c_abs(S.x) + c_abs(S.y) + c_abs(S.z));
      if (dx * dx + dy * dy + dz * dz < lim * lim) mk |= 1ull << j;
    }
    if (ob.prims() && (mk & ~sphere_bits(ob, j0))) mk = prim_exact_cull(ob, j0, mk, m[0], m[1], m[2], half, lsum);
    mask[i] = mk;
  }
}

// Second level: the samples k0..k1 of segment i (arc fractions k / n_b) lie within
// (k1 - k0) L_i / (2 n_b) of the point at fraction (k0 + k1) / (2 n_b); of the candidates `cand`
// (bits relative to j0) those within that radius + reach of it, with the same rounding margin.
constexpr int kCullGroup = 4;  // backbone samples per second-level ball
template <typename T, int N>
CR_HD uint64_t group_sphere_mask(const RobotK<T>& rb, const Chain<T, N>& ch, int i, int k0, int k1,
                                 ObsK<T> ob, int j0, uint64_t cand) {
  const Sphere4<T>* sph = ob.s;
  T lsum = T(0);
#pragma unroll
  for (int l = 0; l < N; ++l) lsum += ch.L[l];
  const T inb = c_div(T(1), T(rb.nb));
  T q[3], m[3], s, c;
  backbone_point(ch.Rb[i], ch.pb[i], ch.ax[i], ch.ay[i], ch.x[i], ch.L[i], T(0.5) * T(k0 + k1) * inb, q, m, s, c);
  const T rad = T(0.5) * T(k1 - k0) * ch.L[i] * inb;
  uint64_t out = 0;
  for (uint64_t b = cand; b; b &= b - 1) {
    const int jj = __ffsll((long long)b) - 1;
    const Sphere4<T> S = sph[j0 + jj];
    const T dx = m[0] - S.x, dy = m[1] - S.y, dz = m[2] - S.z;
    const T lim = rad + S.reach + T(1e-4) * (lsum + S.reach + c_abs(S.x) + c_abs(S.y) + c_abs(S.z));
    if (dx * dx + dy * dy + dz * dz < lim * lim) out |= 1ull << jj;
  }
  if (ob.prims() && (out & ~sphere_bits(ob, j0))) out = prim_exact_cull(ob, j0, out, m[0], m[1], m[2], rad, lsum);
  return out;
}

// The same sets computed by a warp: lane l tests spheres j0 + l and j0 + l + 32 against every
// segment and the ballots assemble the masks (identical in all lanes afterwards).
template <typename T, int N>
__device__ void warp_segment_sphere_masks(const RobotK<T>& rb, const Chain<T, N>& ch, ObsK<T> ob, int j0,
                                          int cnt, uint64_t (&mask)[N]) {
  const Sphere4<T>* sph = ob.s;
  const int lane = threadIdx.x & 31;
  T lsum = T(0);
#pragma unroll
  for (int i = 0; i < N; ++i) lsum += ch.L[i];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    T q[3], m[3], s, c;
    backbone_point(ch.Rb[i], ch.pb[i], ch.ax[i], ch.ay[i], ch.x[i], ch.L[i], T(0.5), q, m, s, c);
    const T half = T(0.5) * ch.L[i];
    uint64_t mk = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = lane + 32 * h;
      bool hit = false;
      if (j < cnt) {
        const Sphere4<T> S = sph[j0 + j];
        const T dx = m[0] - S.x, dy = m[1] - S.y, dz = m[2] - S.z;
        const T lim = half + S.reach + T(1e-4) * (lsum + S.reach + c_abs(S.x) + c_abs(S.y) + c_abs(S.z));
        hit = dx * dx + dy * dy + dz * dz < lim * lim;
      }
      mk |= (uint64_t)__ballot_sync(0xffffffffu, hit) << (32 * h);
    }
    if (ob.prims() && (mk & ~sphere_bits(ob, j0))) mk = prim_exact_cull(ob, j0, mk, m[0], m[1], m[2], half, lsum);
    mask[i] = mk;
  }
}

// ------------------------------------------------------------------------------------------------
// Cost and adjoint of one state, in two phases
// ------------------------------------------------------------------------------------------------
// Per-segment aggregates of the clearance rows for the reverse sweep: G, M = force and moment (about
// the origin) of the segment's own samples, Dx / Dy / DL = their direct terms in (ax, ay, L).
template <typename T, int N> struct StateAgg {
  T G[N][3], M[N][3], Dx[N], Dy[N], DL[N];
};

// A force gw (dF/dw) at the backbone sample of arc fraction sg of segment i (local point q, world point
// wp, segment coefficients s, c of the sub-arc): its share of the segment's force / moment sums and of
// the direct terms in (ax_i, ay_i, L_i), as the sphere rows below accumulate them.
template <typename T, int N, bool PGRAD, int MODEL>
CR_HD void agg_sample_force(const Chain<T, N>& ch, int i, T sg, const T (&q)[3], const T (&wp)[3], T s, T c,
                            const T (&gw)[3], StateAgg<T, N>& ag) {
  ag.G[i][0] += gw[0]; ag.G[i][1] += gw[1]; ag.G[i][2] += gw[2];
  T mw[3];
  cross(wp, gw, mw);
  ag.M[i][0] += mw[0]; ag.M[i][1] += mw[1]; ag.M[i][2] += mw[2];
  T gl[3];
  matTvec(ch.Rb[i], gw, gl);
  T s3, cp;
  seg_deriv(sg * sg * ch.x[i], s, c, s3, cp);
  T dd[2][3], wl[2][3];
  seg_local_derivs(sg * ch.ax[i], sg * ch.ay[i], s, c, s3, cp, sg * ch.L[i], dd, wl);
  ag.Dx[i] += sg * (gl[0] * dd[0][0] + gl[1] * dd[0][1] + gl[2] * dd[0][2]);
  ag.Dy[i] += sg * (gl[0] * dd[1][0] + gl[1] * dd[1][1] + gl[2] * dd[1][2]);
  if (PGRAD || MODEL == CR_MODEL_ARC) ag.DL[i] += (gl[0] * q[0] + gl[1] * q[1] + gl[2] * q[2]) / ch.L[i];
}

// Self-contact rows (Eq. ik_coll's minimum distance over the robot itself, Sec. IV-A; the rows are
// defined for backbone samples a of segment i and b of segment j >= i + 2, adjacent segments meeting
// at a joint): sqrt(rho_s) max(0, gap - |p_a - p_b|), gap = 2 r_body + delta. Adds 1/2 r^2 to coll
// and, when GRAD, equal and opposite forces at the two samples to the segments' aggregates, which
// the reverse sweep turns into the gradient like any sample force. Broad phase: every sample of
// segment i lies within L_i / 2 of its mid-arc point (unit speed in arc length), so a segment pair
// whose mid-arc points are farther apart than (L_i + L_j) / 2 + gap has no active row, nor a sample
// of i farther than L_j / 2 + gap from segment j's; both tests carry the 1e-4 rounding margin of the
// sphere culling. The rows' order and values are the oracle's; only pairs within gap contribute.
template <typename T, int N, bool GRAD, bool PGRAD, int MODEL>
CR_HD void self_contact_forward(const RobotK<T>& rb, const WeightsK<T>& w, const Chain<T, N>& ch,
                                StateAgg<T, N>& ag, T& coll) {
  if (N < 3 || !(w.rho_s > T(0))) return;
  const T gap = T(2) * rb.rbody + w.delta;
  const T inb = c_div(T(1), T(rb.nb));
  T lsum = T(0);
#pragma unroll
  for (int i = 0; i < N; ++i) lsum += ch.L[i];
  const T marg = T(1e-4) * (lsum + gap);
  T mid[N][3];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    T q[3], s, c;
    backbone_point(ch.Rb[i], ch.pb[i], ch.ax[i], ch.ay[i], ch.x[i], ch.L[i], T(0.5), q, mid[i], s, c);
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
#pragma unroll
    for (int j = i + 2; j < N; ++j) {
      {
        const T dx = mid[i][0] - mid[j][0], dy = mid[i][1] - mid[j][1], dz = mid[i][2] - mid[j][2];
        const T lim = T(0.5) * (ch.L[i] + ch.L[j]) + gap + marg;
        if (!(dx * dx + dy * dy + dz * dz < lim * lim)) continue;
      }
      const T limj = T(0.5) * ch.L[j] + gap + marg;
      for (int ka = 1; ka <= rb.nb; ++ka) {
        const T sa = T(ka) * inb;
        T qa[3], pa[3], s_a, c_a;
        backbone_point(ch.Rb[i], ch.pb[i], ch.ax[i], ch.ay[i], ch.x[i], ch.L[i], sa, qa, pa, s_a, c_a);
        {
          const T ex = pa[0] - mid[j][0], ey = pa[1] - mid[j][1], ez = pa[2] - mid[j][2];
          if (!(ex * ex + ey * ey + ez * ez < limj * limj)) continue;
        }
        T ga[3] = {T(0), T(0), T(0)};
        bool hit = false;
        for (int kb = 1; kb <= rb.nb; ++kb) {
          const T sb = T(kb) * inb;
          T qb[3], pb[3], s_b, c_b;
          backbone_point(ch.Rb[j], ch.pb[j], ch.ax[j], ch.ay[j], ch.x[j], ch.L[j], sb, qb, pb, s_b, c_b);
          const T dx = pa[0] - pb[0], dy = pa[1] - pb[1], dz = pa[2] - pb[2];
          const T d2 = dx * dx + dy * dy + dz * dz;
          if (!(d2 < gap * gap)) continue;
          const T dist = c_sqrt(d2);
          const T viol = gap - dist;
          const T rr = w.ss * viol;
          coll += T(0.5) * rr * rr;
          if (GRAD) {
            const T f = -w.rho_s * viol / dist;
            const T gw[3] = {f * dx, f * dy, f * dz};  // dF/dp_a; p_b takes -gw
            ga[0] += gw[0]; ga[1] += gw[1]; ga[2] += gw[2];
            const T gb[3] = {-gw[0], -gw[1], -gw[2]};
            agg_sample_force<T, N, PGRAD, MODEL>(ch, j, sb, qb, pb, s_b, c_b, gb, ag);
            hit = true;
          }
        }
        if (GRAD && hit) agg_sample_force<T, N, PGRAD, MODEL>(ch, i, sa, qa, pa, s_a, c_a, ga, ag);
      }
    }
  }
}

// Forward phase: chain, clearance rows (and their aggregates when GRAD), and the penalty rows on u
// (bounds, sum-zero, curvature). Returns their part of F; *coll_out = the clearance part.
// BOX = false leaves out the bound and sum-zero rows: on the feasible set {|u_j| <= b, sum u_j = 0}
// they vanish, so callers whose state was just projected onto it skip them (in FP32 the sum-zero
// row would only add the rounding residue of the projection). OBST compiles the collision rows:
// the spheres' and, with w.rho_s > 0, the self-contact rows (with_self = false leaves the latter to
// another thread that evaluates the same state).
template <typename T, int N, bool OBST, bool GRAD, bool PGRAD, bool BOX = true, int MODEL = CR_MODEL_TENDON>
CR_HD T state_forward(const RobotK<T>& rb, const WeightsK<T>& w, ObsK<T> ob, int no,
                      const T (&u)[3 * N], Chain<T, N>& ch, StateAgg<T, N>& ag, T* coll_out,
                      bool with_self = true) {
  const Sphere4<T>* sph = ob.s;
  chain_forward<T, N, MODEL>(rb, u, ch);
  T coll = T(0);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    ag.G[i][0] = ag.G[i][1] = ag.G[i][2] = T(0);
    ag.M[i][0] = ag.M[i][1] = ag.M[i][2] = T(0);
    ag.Dx[i] = ag.Dy[i] = ag.DL[i] = T(0);
  }
  if (OBST && no > 0) {
    const T inb = T(1) / T(rb.nb);
    for (int j0 = 0; j0 < no; j0 += 64) {
    uint64_t mk[N];
    segment_sphere_masks(rb, ch, ob, j0, no - j0 < 64 ? no - j0 : 64, mk);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      if (!mk[i]) continue;
      for (int k0 = 1; k0 <= rb.nb; k0 += kCullGroup) {
      const int k1 = k0 + kCullGroup - 1 < rb.nb ? k0 + kCullGroup - 1 : rb.nb;
      const uint64_t gm = group_sphere_mask<T, N>(rb, ch, i, k0, k1, ob, j0, mk[i]);
      if (!gm) continue;
      for (int k = k0; k <= k1; ++k) {
        T sg = T(k) * inb;
        T q[3], wp[3], s, c;
        backbone_point(ch.Rb[i], ch.pb[i], ch.ax[i], ch.ay[i], ch.x[i], ch.L[i], sg, q, wp, s, c);
        T gw[3] = {T(0), T(0), T(0)};
        bool hit = false;
        const uint64_t sb = sphere_bits(ob, j0);
        for (uint64_t bits = gm & sb; bits; bits &= bits - 1) {
          Sphere4<T> S = sph[j0 + __ffsll((long long)bits) - 1];
          T dx = wp[0] - S.x, dy = wp[1] - S.y, dz = wp[2] - S.z;
          T d2 = dx * dx + dy * dy + dz * dz;
          if (d2 < S.reach * S.reach) {
            T dist = c_sqrt(d2);
            T viol = S.reach - dist;
            T rr = w.sc * viol;
            coll += T(0.5) * rr * rr;
            if (GRAD) {
              T f = -w.rho_c * viol / dist;
              gw[0] += f * dx; gw[1] += f * dy; gw[2] += f * dz;
              hit = true;
            }
          }
        }
        for (uint64_t bits = ob.prims() ? gm & ~sb : 0ull; bits; bits &= bits - 1) {  // primitives: sd(x) rows
          const PrimK<T>& P = ob.p[j0 + __ffsll((long long)bits) - 1 - ob.ns];
          T viol, nv[3];
          if (prim_active(P, wp, P.reach, viol, nv)) {
            T rr = w.sc * viol;
            coll += T(0.5) * rr * rr;
            if (GRAD) {
              T f = -w.rho_c * viol;
              gw[0] += f * nv[0]; gw[1] += f * nv[1]; gw[2] += f * nv[2];
              hit = true;
            }
          }
        }
        if (GRAD && hit) {
          ag.G[i][0] += gw[0]; ag.G[i][1] += gw[1]; ag.G[i][2] += gw[2];
          T mw[3];
          cross(wp, gw, mw);
          ag.M[i][0] += mw[0]; ag.M[i][1] += mw[1]; ag.M[i][2] += mw[2];
          T gl[3];
          matTvec(ch.Rb[i], gw, gl);
          T axs = sg * ch.ax[i], ays = sg * ch.ay[i];
          T s3, cp;
          seg_deriv(sg * sg * ch.x[i], s, c, s3, cp);
          T dd[2][3], wl[2][3];
          seg_local_derivs(axs, ays, s, c, s3, cp, sg * ch.L[i], dd, wl);
          ag.Dx[i] += sg * (gl[0] * dd[0][0] + gl[1] * dd[0][1] + gl[2] * dd[0][2]);
          ag.Dy[i] += sg * (gl[0] * dd[1][0] + gl[1] * dd[1][1] + gl[2] * dd[1][2]);
          if (PGRAD || MODEL == CR_MODEL_ARC) ag.DL[i] += (gl[0] * q[0] + gl[1] * q[1] + gl[2] * q[2]) / ch.L[i];
        }
      }
      }
    }
    }
  }
  if (OBST && with_self) self_contact_forward<T, N, GRAD, PGRAD, MODEL>(rb, w, ch, ag, coll);
  if (coll_out) *coll_out = coll;
  T F = coll;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if (BOX && MODEL == CR_MODEL_ARC) {  // length bounds of the extendable segment
      T hi = ch.L[i] - rb.lmax[i], lo = rb.lmin[i] - ch.L[i];
      if (hi > T(0)) F += T(0.5) * w.rho_b * hi * hi;
      if (lo > T(0)) F += T(0.5) * w.rho_b * lo * lo;
    } else if (BOX) {
      T su = u[3 * i] + u[3 * i + 1] + u[3 * i + 2];
      F += T(0.5) * w.rho_eq * su * su;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        T hi = u[3 * i + j] - rb.umax[i], lo = -rb.umax[i] - u[3 * i + j];
        if (hi > T(0)) F += T(0.5) * w.rho_b * hi * hi;
        if (lo > T(0)) F += T(0.5) * w.rho_b * lo * lo;
      }
    }
    // in the arc model theta <= theta_max is part of the projected set, so the curvature row too
    // vanishes where BOX = false
    if ((BOX || MODEL != CR_MODEL_ARC) && ch.x[i] > rb.thmax[i] * rb.thmax[i]) {
      T vk = c_sqrt(ch.x[i]) - rb.thmax[i];
      F += T(0.5) * w.rho_k * vk * vk;
    }
  }
  return F;
}

// Reverse phase: given dF/dp at the tip (Ftip) and the world moment of dF/d(tip rotation) (Rtip),
// sweep the segments from the tip to the base: the force and moment of everything downstream of
// segment i act on (ax_i, ay_i) through the segment's local derivatives. Adds the penalty gradients
// and writes dF/du (and dF/dL, dF/dr_c when PGRAD). BOX as in state_forward. In the arc model the
// state's own lengths take the place of dF/du_i2 (dF/dL_i: everything beyond the segment's end moves
// with d_i, its own samples scale with L_i). The moment is kept about the end point of the current
// segment (moved to the next one by (p_end - p_base) x F), so no large moment about the origin is
// formed and cancelled. AGG = false: the state has no clearance rows (its aggregates are zero).
template <typename T, int N, bool PGRAD, bool BOX = true, int MODEL = CR_MODEL_TENDON, bool AGG = true>
CR_HD void state_reverse(const RobotK<T>& rb, const WeightsK<T>& w, const T (&u)[3 * N], const Chain<T, N>& ch,
                         const StateAgg<T, N>& ag, const T (&Ftip)[3], const T (&Rtip)[3], T (&gu)[3 * N], T* gL,
                         T* grc) {
  T Fs[3] = {Ftip[0], Ftip[1], Ftip[2]};
  T Mp[3] = {Rtip[0], Rtip[1], Rtip[2]};  // moment about the end point of segment i (the tip force acts there)
  T gnext[3] = {T(0), T(0), T(0)};  // coupled routing: the u-space gradient of segment i + 1
#pragma unroll
  for (int i = N - 1; i >= 0; --i) {
    T Fl[3], Ml[3];
    if (i == 0) {  // the base frame is the identity
#pragma unroll
      for (int a = 0; a < 3; ++a) { Fl[a] = Fs[a]; Ml[a] = Mp[a]; }
    } else {
      matTvec(ch.Rb[i], Fs, Fl);
      matTvec(ch.Rb[i], Mp, Ml);
    }
    T s3, cp;
    seg_deriv(ch.x[i], ch.s[i], ch.c[i], s3, cp);
    // Fl . d(d_i)/da_k + Ml . J_l dw/da_k, the products of seg_local_derivs written out:
    // with Fa = a . Fl_xy, Ma = a . Ml_xy and cf = cp Fa + sp Fl_z,
    // gx = L (c Fl_x + 2 ax cf) + Ml_y - s3 ay Ma - c ay Ml_z,
    // gy = L (c Fl_y + 2 ay cf) - Ml_x + s3 ax Ma + c ax Ml_z.
    const T ax = ch.ax[i], ay = ch.ay[i], cc = ch.c[i], L = ch.L[i];
    T sp = T(0.5) * (s3 - cc);
    T Fa = ax * Fl[0] + ay * Fl[1], Ma = ax * Ml[0] + ay * Ml[1];
    T cf = cp * Fa + sp * Fl[2];
    T gx = L * (cc * Fl[0] + T(2) * ax * cf) + Ml[1] - s3 * ay * Ma - cc * ay * Ml[2];
    T gy = L * (cc * Fl[1] + T(2) * ay * cf) - Ml[0] + s3 * ax * Ma + cc * ax * Ml[2];
    if (AGG) {
      gx += ag.Dx[i];
      gy += ag.Dy[i];
    }
    if ((BOX || MODEL != CR_MODEL_ARC) && ch.x[i] > rb.thmax[i] * rb.thmax[i]) {
      T th = c_sqrt(ch.x[i]);
      T f = w.rho_k * (th - rb.thmax[i]) / th;
      gx += f * ch.ax[i];
      gy += f * ch.ay[i];
    }
    T g0, g1, g2;
    bend_cols<MODEL>(rb, i, gx, gy, g0, g1, g2);
    T gj[3] = {g0, g1, g2};
    if (MODEL == CR_MODEL_COUPLED) {  // dF/dq_i = dF/du_i - dF/du_{i+1} (u = D q)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const T gu_ij = gj[j];
        gj[j] = gu_ij - gnext[j];
        gnext[j] = gu_ij;
      }
    }
    const T DLi = AGG ? ag.DL[i] : T(0);
    if (MODEL == CR_MODEL_ARC) {
      const T di[3] = {ch.L[i] * ch.c[i] * ch.ax[i], ch.L[i] * ch.c[i] * ch.ay[i], ch.L[i] * ch.s[i]};
      T gl = (Fl[0] * di[0] + Fl[1] * di[1] + Fl[2] * di[2]) / ch.L[i];
      if (AGG) gl += DLi;
      if (BOX) {
        T hi = ch.L[i] - rb.lmax[i], lo = rb.lmin[i] - ch.L[i];
        gl += (hi > T(0) ? w.rho_b * hi : T(0)) - (lo > T(0) ? w.rho_b * lo : T(0));
      }
      gu[3 * i] = gj[0];
      gu[3 * i + 1] = gj[1];
      gu[3 * i + 2] = gl;
    } else if (BOX) {
      T su = u[3 * i] + u[3 * i + 1] + u[3 * i + 2];
      T geq = w.rho_eq * su;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        T uj = u[3 * i + j];
        T hi = uj - rb.umax[i], lo = -rb.umax[i] - uj;
        T gb = (hi > T(0) ? w.rho_b * hi : T(0)) - (lo > T(0) ? w.rho_b * lo : T(0));
        gu[3 * i + j] = gj[j] + geq + gb;
      }
    } else {
#pragma unroll
      for (int j = 0; j < 3; ++j) gu[3 * i + j] = gj[j];
    }
    if (PGRAD) {
      // dF/dL_i: translation d_i = L (...) scales with L; own samples q scale with L too
      T di[3] = {ch.L[i] * ch.c[i] * ch.ax[i], ch.L[i] * ch.c[i] * ch.ay[i], ch.L[i] * ch.s[i]};
      gL[i] = (Fl[0] * di[0] + Fl[1] * di[1] + Fl[2] * di[2]) / ch.L[i];
      if (AGG) gL[i] += DLi;
      // dF/dr_c,i: a = K(...) with K = -2/(3 r_c) so da/dr_c = -a / r_c
      grc[i] = -(ch.ax[i] * gx + ch.ay[i] * gy) / rb.rc[i];
    }
    if (i > 0) {
      // to the base of segment i (the end of segment i - 1): M <- M + (p_end - p_base) x F, then the
      // segment's own samples: force G_i, moment about the base M_i - p_base x G_i (M_i about the origin)
      T dp[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) dp[a] = ((i == N - 1) ? ch.p[a] : ch.pb[(i + 1 < N) ? i + 1 : i][a]) - ch.pb[i][a];
      T dm[3];
      cross(dp, Fs, dm);
      Mp[0] += dm[0]; Mp[1] += dm[1]; Mp[2] += dm[2];
      if (AGG) {
        T bg[3];
        cross(ch.pb[i], ag.G[i], bg);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          Mp[a] += ag.M[i][a] - bg[a];
          Fs[a] += ag.G[i][a];
        }
      }
    }
  }
}

// Tip force and moment of the pose rows: dF/dp = w_p^2 (p - p_t); for IK6 the rotation term is
// w_R^2 R e (the inverse right Jacobian leaves e unchanged), for IK5 (F = 1/2 w_R^2 |z - z_t|^2) it is
// w_R^2 z_t x z.
template <typename T>
CR_HD void pose_tip_force(int kind, const WeightsK<T>& w, const TargetK<T>& tg, const T (&R)[9], const T (&r)[6],
                          const T (&e)[3], T (&Ftip)[3], T (&Rtip)[3]) {
  Ftip[0] = w.wp * r[0];
  Ftip[1] = w.wp * r[1];
  Ftip[2] = w.wp * r[2];
  if (kind == CR_TASK_IK5) {
    T z[3] = {R[2], R[5], R[8]};
    T zt[3] = {tg.R[0], tg.R[1], tg.R[2]};
    T cz[3];
    cross(zt, z, cz);
    Rtip[0] = w.wR2 * cz[0]; Rtip[1] = w.wR2 * cz[1]; Rtip[2] = w.wR2 * cz[2];
  } else {
    T re[3];
    matvec(R, e, re);
    Rtip[0] = w.wR2 * re[0]; Rtip[1] = w.wR2 * re[1]; Rtip[2] = w.wR2 * re[2];
  }
}

// Cost (and adjoint) of an IK state: the two phases around the pose rows. BOX as in state_forward.
template <typename T, int N, bool OBST, bool GRAD, bool PGRAD, bool BOX = true, int MODEL = CR_MODEL_TENDON>
CR_HD T eval_ik(const RobotK<T>& rb, const WeightsK<T>& w, int kind, const TargetK<T>& tg,
                ObsK<T> sph, int no, const T (&u)[3 * N], T (&gu)[3 * N], T* gL, T* grc,
                T* coll_out) {
  Chain<T, N> ch;
  StateAgg<T, N> ag;
  T F = state_forward<T, N, OBST, GRAD, PGRAD, BOX, MODEL>(rb, w, sph, no, u, ch, ag, coll_out);
  T r[6], e[3], ang, sn, cs;
  pose_rows(kind, w, tg, ch.R, ch.p, r, e, ang, sn, cs);
  F += T(0.5) * (r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3] + r[4] * r[4] + r[5] * r[5]);
  if (!GRAD) return F;
  T Ftip[3], Rtip[3];
  pose_tip_force(kind, w, tg, ch.R, r, e, Ftip, Rtip);
  state_reverse<T, N, PGRAD, BOX, MODEL, OBST>(rb, w, u, ch, ag, Ftip, Rtip, gu, gL, grc);
  return F;
}

// ------------------------------------------------------------------------------------------------
// Tip Jacobian (world twists of every segment)
// ------------------------------------------------------------------------------------------------
// tw[i][k] = (v, w): a point p rigidly downstream of segment i moves by v + w x p per unit da_k.
template <typename T, int N>
CR_HD void segment_twists(const RobotK<T>& rb, const Chain<T, N>& ch, T (&tv)[N][2][3], T (&tw)[N][2][3]) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    T s3, cp;
    seg_deriv(ch.x[i], ch.s[i], ch.c[i], s3, cp);
    T dd[2][3], wl[2][3];
    seg_local_derivs(ch.ax[i], ch.ay[i], ch.s[i], ch.c[i], s3, cp, ch.L[i], dd, wl);
    T Pend[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) Pend[a] = (i == N - 1) ? ch.p[a] : ch.pb[(i + 1 < N) ? i + 1 : i][a];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      T wv[3], dv[3];
      matvec(ch.Rb[i], wl[k], wv);
      matvec(ch.Rb[i], dd[k], dv);
      T wP[3];
      cross(wv, Pend, wP);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        tw[i][k][a] = wv[a];
        tv[i][k][a] = dv[a] - wP[a];
      }
    }
  }
}

// Arc model: translation of everything beyond segment i per unit length, Rb_i (c a_x, c a_y, s)
// (d_i is proportional to L_i; the segment's rotation does not depend on it).
template <typename T, int N>
CR_HD void length_dir(const Chain<T, N>& ch, int i, T (&v)[3]) {
  const T d[3] = {ch.c[i] * ch.ax[i], ch.c[i] * ch.ay[i], ch.s[i]};
  matvec(ch.Rb[i], d, v);
}

// Tip Jacobian in state space: Jp[a][q] = dp_a/du_q, Jw[a][q] = world angular velocity.
template <typename T, int N, int MODEL = CR_MODEL_TENDON>
CR_HD void tip_jacobian(const RobotK<T>& rb, const Chain<T, N>& ch, T (&Jp)[3][3 * N], T (&Jw)[3][3 * N]) {
  T tv[N][2][3], tw[N][2][3];
  segment_twists(rb, ch, tv, tw);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    T jp[2][3], jw[2][3];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      T wp[3];
      cross(tw[i][k], ch.p, wp);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        jp[k][a] = tv[i][k][a] + wp[a];
        jw[k][a] = tw[i][k][a];
      }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      bend_cols<MODEL>(rb, i, jp[0][a], jp[1][a], Jp[a][3 * i], Jp[a][3 * i + 1], Jp[a][3 * i + 2]);
      bend_cols<MODEL>(rb, i, jw[0][a], jw[1][a], Jw[a][3 * i], Jw[a][3 * i + 1], Jw[a][3 * i + 2]);
    }
    if (MODEL == CR_MODEL_ARC) {
      T v[3];
      length_dir(ch, i, v);
#pragma unroll
      for (int a = 0; a < 3; ++a) Jp[a][3 * i + 2] = v[a];
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    to_actuator<MODEL, T, N>(Jp[a]);
    to_actuator<MODEL, T, N>(Jw[a]);
  }
}

// ------------------------------------------------------------------------------------------------
// LM normal equations of an IK state: A = J^T J (packed lower), g = J^T r, F = 1/2 |r|^2.
// J and r in T; accumulation in TA.
// ------------------------------------------------------------------------------------------------
CR_HD constexpr int tri(int i, int j) { return i * (i + 1) / 2 + j; }  // i >= j

// Two-float accumulator for the normal equations of the FP32 bulk form. J^T J of an FP32 Jacobian
// with condition number kappa, rounded to FP32, carries a relative error of about kappa^2 eps32 in
// its small eigendirections, which the LM step inherits (measured: step errors of 5e-5 of the
// displacement bound at kappa(J) = 400, against 2e-8 from the rounding of J and r alone). FP64
// accumulation would avoid that on the FP64 pipe (1/64 of the FP32 rate on this GPU); instead every
// product of two FP32 numbers is split exactly into p + e (p = x y rounded, e = fma(x, y, -p)) and
// added to a (hi, lo) pair with the error-free sum of Knuth (TwoSum), all on the FP32 pipe. The
// explicitly rounded intrinsics keep the compiler from fusing a product into the following sum,
// which would break the exactness. hi + lo carries about 48 bits; it is converted to FP64 for the
// Cholesky.
struct F2 {
  float hi, lo;
  CR_HD F2(float v = 0.0f) : hi(v), lo(0.0f) {}
};
CR_HD void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// acc += v, acc += x y (exact product for F2), generic for float and double accumulators.
template <typename TA, typename T> CR_HD void acc_add(TA& acc, T v) { acc += TA(v); }
template <typename TA, typename T> CR_HD void acc_prod(TA& acc, T x, T y) { acc += TA(x) * TA(y); }
template <> CR_HD void acc_add<F2, float>(F2& acc, float v) {
  float s, e;
  two_sum(acc.hi, v, s, e);
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, e);
}
template <> CR_HD void acc_prod<F2, float>(F2& acc, float x, float y) {
  const float p = __fmul_rn(x, y);
  const float pe = fmaf(x, y, -p);  // x y - p, exact
  float s, e;
  two_sum(acc.hi, p, s, e);
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(e, pe));
}
CR_HD double to_f64(float v) { return double(v); }
CR_HD double to_f64(double v) { return v; }
CR_HD double to_f64(const F2& v) { return double(v.hi) + double(v.lo); }
// The accumulator of an LM normal matrix for bulk precision T.
template <typename T> struct NormalAcc { typedef T type; };
template <> struct NormalAcc<float> { typedef F2 type; };

// A is any indexable packed lower triangle (normally a register array).
template <typename TA, int D, typename T, typename AArr>
CR_HD void rank1(AArr&& A, TA (&g)[D], const T (&j)[D], T r) {
#pragma unroll
  for (int a = 0; a < D; ++a) {
    acc_prod(g[a], j[a], r);
#pragma unroll
    for (int b = 0; b <= a; ++b) acc_prod(A[tri(a, b)], j[a], j[b]);
  }
}

// Adds scale * n . dp/du of the backbone sample at arc fraction sg of segment i (local point q, world
// point wp, sub-arc coefficients s, c) to the row jr: segments l < i move it rigidly (twist plus, in
// the arc model, the length direction), segment i through its own sub-arc.
template <typename T, int N, int MODEL>
CR_HD void add_sample_row(const RobotK<T>& rb, const Chain<T, N>& ch, const T (&tv)[N][2][3], const T (&tw)[N][2][3],
                          const T (&ldir)[N][3], int i, T sg, const T (&q)[3], const T (&wp)[3], T s, T c,
                          const T (&nh)[3], T scale, T (&jr)[3 * N]) {
#pragma unroll
  for (int l = 0; l < N; ++l) {
    if (l > i) break;
    T ga[2], gl = T(0);
    if (l < i) {
      if (MODEL == CR_MODEL_ARC) gl = scale * (nh[0] * ldir[l][0] + nh[1] * ldir[l][1] + nh[2] * ldir[l][2]);
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        T wx[3];
        cross(tw[l][kk], wp, wx);
        ga[kk] = scale * (nh[0] * (tv[l][kk][0] + wx[0]) + nh[1] * (tv[l][kk][1] + wx[1]) +
                          nh[2] * (tv[l][kk][2] + wx[2]));
      }
    } else {
      T s3, cp;
      seg_deriv(sg * sg * ch.x[i], s, c, s3, cp);
      T dd[2][3], wl[2][3];
      seg_local_derivs(sg * ch.ax[i], sg * ch.ay[i], s, c, s3, cp, sg * ch.L[i], dd, wl);
      T nl[3];
      matTvec(ch.Rb[i], nh, nl);
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) ga[kk] = scale * sg * (nl[0] * dd[kk][0] + nl[1] * dd[kk][1] + nl[2] * dd[kk][2]);
      if (MODEL == CR_MODEL_ARC) gl = scale * (nl[0] * q[0] + nl[1] * q[1] + nl[2] * q[2]) / ch.L[i];
    }
    T c0, c1, c2;
    bend_cols<MODEL>(rb, l, ga[0], ga[1], c0, c1, c2);
    jr[3 * l] += c0;
    jr[3 * l + 1] += c1;
    jr[3 * l + 2] += MODEL == CR_MODEL_ARC ? gl : c2;
  }
}

template <typename T, typename TA, int N, bool OBST, int MODEL = CR_MODEL_TENDON, typename AArr>
CR_HD T eval_ik_normal(const RobotK<T>& rb, const WeightsK<T>& w, int kind, const TargetK<T>& tg,
                       ObsK<T> ob, int no, const T (&u)[3 * N], AArr&& A, TA (&g)[3 * N]) {
  constexpr int D = 3 * N;
  const Sphere4<T>* sph = ob.s;
#pragma unroll
  for (int a = 0; a < D * (D + 1) / 2; ++a) A[a] = TA(0);
#pragma unroll
  for (int a = 0; a < D; ++a) g[a] = TA(0);
  Chain<T, N> ch;
  chain_forward<T, N, MODEL>(rb, u, ch);
  T r[6], e[3], ang, sn, cs;
  pose_rows(kind, w, tg, ch.R, ch.p, r, e, ang, sn, cs);
  T F = T(0.5) * (r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3] + r[4] * r[4] + r[5] * r[5]);
  T tv[N][2][3], tw[N][2][3];
  segment_twists(rb, ch, tv, tw);
  // tip Jacobian in u-space
  T Jp[3][D], Jw[3][D];
#pragma unroll
  for (int i = 0; i < N; ++i) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      T wp0[3], wp1[3];
      cross(tw[i][0], ch.p, wp0);
      cross(tw[i][1], ch.p, wp1);
      bend_cols<MODEL>(rb, i, tv[i][0][a] + wp0[a], tv[i][1][a] + wp1[a], Jp[a][3 * i],
                       Jp[a][3 * i + 1], Jp[a][3 * i + 2]);
      bend_cols<MODEL>(rb, i, tw[i][0][a], tw[i][1][a], Jw[a][3 * i], Jw[a][3 * i + 1],
                       Jw[a][3 * i + 2]);
    }
  }
  T ldir[N][3];  // arc model: d(point beyond segment i) / dL_i
  if (MODEL == CR_MODEL_ARC) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      length_dir(ch, i, ldir[i]);
#pragma unroll
      for (int a = 0; a < 3; ++a) Jp[a][3 * i + 2] = ldir[i][a];
    }
  }
  // position rows
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    T jr[D];
#pragma unroll
    for (int q = 0; q < D; ++q) jr[q] = w.wp * Jp[a][q];
    to_actuator<MODEL, T, N>(jr);
    rank1<TA, D>(A, g, jr, r[a]);
  }
  // rotation rows
  T Mrot[3][3];  // rows of d e / d(world rotation)
  if (kind == CR_TASK_IK5) {
    // d(z - z_t) = w x z = -[z]x w
    T z0 = ch.R[2], z1 = ch.R[5], z2 = ch.R[8];
    Mrot[0][0] = T(0);  Mrot[0][1] = z2;    Mrot[0][2] = -z1;
    Mrot[1][0] = -z2;   Mrot[1][1] = T(0);  Mrot[1][2] = z0;
    Mrot[2][0] = z1;    Mrot[2][1] = -z0;   Mrot[2][2] = T(0);
  } else {
    // de = J_r^-1(e) R^T dw, J_r^-1(e) = I + [e]x/2 + beta [e]x^2
    T be = log_beta(ang);
    T E2[3][3] = {{-(e[1] * e[1] + e[2] * e[2]), e[0] * e[1], e[0] * e[2]},
                  {e[0] * e[1], -(e[0] * e[0] + e[2] * e[2]), e[1] * e[2]},
                  {e[0] * e[2], e[1] * e[2], -(e[0] * e[0] + e[1] * e[1])}};
    T Jr[3][3] = {{T(1) + be * E2[0][0], T(-0.5) * e[2] + be * E2[0][1], T(0.5) * e[1] + be * E2[0][2]},
                  {T(0.5) * e[2] + be * E2[1][0], T(1) + be * E2[1][1], T(-0.5) * e[0] + be * E2[1][2]},
                  {T(-0.5) * e[1] + be * E2[2][0], T(0.5) * e[0] + be * E2[2][1], T(1) + be * E2[2][2]}};
    // Mrot = Jr R^T
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
        Mrot[a][b] = Jr[a][0] * ch.R[3 * b] + Jr[a][1] * ch.R[3 * b + 1] + Jr[a][2] * ch.R[3 * b + 2];
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    T jr[D];
#pragma unroll
    for (int q = 0; q < D; ++q)
      jr[q] = w.wR * (Mrot[a][0] * Jw[0][q] + Mrot[a][1] * Jw[1][q] + Mrot[a][2] * Jw[2][q]);
    to_actuator<MODEL, T, N>(jr);
    rank1<TA, D>(A, g, jr, r[3 + a]);
  }
  // bounds (single-entry rows), sum-zero (segment block of ones), curvature (segment rank-1)
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if (MODEL == CR_MODEL_ARC) {  // length bounds: single-entry rows on the length column
      const int q = 3 * i + 2;
      T hi = ch.L[i] - rb.lmax[i], lo = rb.lmin[i] - ch.L[i];
      if (hi > T(0)) { F += T(0.5) * w.rho_b * hi * hi; acc_add(g[q], w.rho_b * hi); acc_add(A[tri(q, q)], w.rho_b); }
      if (lo > T(0)) { F += T(0.5) * w.rho_b * lo * lo; acc_add(g[q], -(w.rho_b * lo)); acc_add(A[tri(q, q)], w.rho_b); }
    } else {
      T su = u[3 * i] + u[3 * i + 1] + u[3 * i + 2];
      F += T(0.5) * w.rho_eq * su * su;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        int q = 3 * i + j;
        acc_add(g[q], w.rho_eq * su);
#pragma unroll
        for (int j2 = 0; j2 <= j; ++j2) acc_add(A[tri(q, 3 * i + j2)], w.rho_eq);
        T hi = u[q] - rb.umax[i], lo = -rb.umax[i] - u[q];
        if (hi > T(0)) { F += T(0.5) * w.rho_b * hi * hi; acc_add(g[q], w.rho_b * hi); acc_add(A[tri(q, q)], w.rho_b); }
        if (lo > T(0)) { F += T(0.5) * w.rho_b * lo * lo; acc_add(g[q], -(w.rho_b * lo)); acc_add(A[tri(q, q)], w.rho_b); }
      }
    }
    if (ch.x[i] > rb.thmax[i] * rb.thmax[i]) {
      T th = c_sqrt(ch.x[i]);
      T vk = th - rb.thmax[i];
      F += T(0.5) * w.rho_k * vk * vk;
      T jx = w.sk * ch.ax[i] / th, jy = w.sk * ch.ay[i] / th;
      T j0, j1, j2;
      bend_cols<MODEL>(rb, i, jx, jy, j0, j1, j2);
      T jj[3] = {j0, j1, j2};
      T rr = w.sk * vk;
      if (MODEL == CR_MODEL_COUPLED) {  // the row reaches segments i and i - 1 through u = D q
        T jr[D];
#pragma unroll
        for (int qq = 0; qq < D; ++qq) jr[qq] = qq / 3 == i ? jj[qq % 3] : T(0);
        to_actuator<MODEL, T, N>(jr);
        rank1<TA, D>(A, g, jr, rr);
      } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          acc_prod(g[3 * i + a], jj[a], rr);
#pragma unroll
          for (int b = 0; b <= a; ++b) acc_prod(A[tri(3 * i + a, 3 * i + b)], jj[a], jj[b]);
        }
      }
    }
  }
  if (OBST && no > 0) {
    const T inb = T(1) / T(rb.nb);
    for (int j0 = 0; j0 < no; j0 += 64) {
    uint64_t mk[N];
    segment_sphere_masks(rb, ch, ob, j0, no - j0 < 64 ? no - j0 : 64, mk);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      if (!mk[i]) continue;
      for (int k0 = 1; k0 <= rb.nb; k0 += kCullGroup) {
      const int k1 = k0 + kCullGroup - 1 < rb.nb ? k0 + kCullGroup - 1 : rb.nb;
      const uint64_t gm = group_sphere_mask<T, N>(rb, ch, i, k0, k1, ob, j0, mk[i]);
      if (!gm) continue;
      for (int k = k0; k <= k1; ++k) {
        T sg = T(k) * inb;
        T q[3], wp[3], s, c;
        backbone_point(ch.Rb[i], ch.pb[i], ch.ax[i], ch.ay[i], ch.x[i], ch.L[i], sg, q, wp, s, c);
        for (uint64_t bits = gm; bits; bits &= bits - 1) {
          const int jo = j0 + __ffsll((long long)bits) - 1;
          T viol, nh[3];
          if (ob.prims() && jo >= ob.ns) {  // a primitive: the same row with sd(x) for the centre distance
            const PrimK<T>& P = ob.p[jo - ob.ns];
            if (!prim_active(P, wp, P.reach, viol, nh)) continue;
          } else {
            Sphere4<T> S = sph[jo];
            T dx = wp[0] - S.x, dy = wp[1] - S.y, dz = wp[2] - S.z;
            T d2 = dx * dx + dy * dy + dz * dz;
            if (!(d2 < S.reach * S.reach)) continue;
            T dist = c_sqrt(d2);
            viol = S.reach - dist;
            nh[0] = dx / dist; nh[1] = dy / dist; nh[2] = dz / dist;
          }
          T rr = w.sc * viol;
          F += T(0.5) * rr * rr;
          // d r / d w = -sqrt(rho_c) n
          T jr[D];
#pragma unroll
          for (int qq = 0; qq < D; ++qq) jr[qq] = T(0);
#pragma unroll
          for (int l = 0; l < N; ++l) {
            if (l > i) break;
            T ga[2], gl = T(0);
            if (l < i) {
              if (MODEL == CR_MODEL_ARC)
                gl = -w.sc * (nh[0] * ldir[l][0] + nh[1] * ldir[l][1] + nh[2] * ldir[l][2]);
#pragma unroll
              for (int kk = 0; kk < 2; ++kk) {
                T wx[3];
                cross(tw[l][kk], wp, wx);
                ga[kk] = -w.sc * (nh[0] * (tv[l][kk][0] + wx[0]) + nh[1] * (tv[l][kk][1] + wx[1]) +
                                  nh[2] * (tv[l][kk][2] + wx[2]));
              }
            } else {
              T s3, cp;
              seg_deriv(sg * sg * ch.x[i], s, c, s3, cp);
              T dd[2][3], wl[2][3];
              seg_local_derivs(sg * ch.ax[i], sg * ch.ay[i], s, c, s3, cp, sg * ch.L[i], dd, wl);
              T nl[3];
              matTvec(ch.Rb[i], nh, nl);
#pragma unroll
              for (int kk = 0; kk < 2; ++kk)
                ga[kk] = -w.sc * sg * (nl[0] * dd[kk][0] + nl[1] * dd[kk][1] + nl[2] * dd[kk][2]);
              if (MODEL == CR_MODEL_ARC)  // the own sample q scales with L_i
                gl = -w.sc * (nl[0] * q[0] + nl[1] * q[1] + nl[2] * q[2]) / ch.L[i];
            }
            bend_cols<MODEL>(rb, l, ga[0], ga[1], jr[3 * l], jr[3 * l + 1], jr[3 * l + 2]);
            if (MODEL == CR_MODEL_ARC) jr[3 * l + 2] = gl;
          }
          to_actuator<MODEL, T, N>(jr);
          rank1<TA, D>(A, g, jr, rr);
        }
      }
      }
    }
    }
  }
  // self-contact rows (as in self_contact_forward): r = sqrt(rho_s) (gap - |p_a - p_b|), its row
  // -sqrt(rho_s) n . (dp_a/du - dp_b/du) with n = (p_a - p_b) / |p_a - p_b|
  if (OBST && N >= 3 && w.rho_s > T(0)) {
    const T gap = T(2) * rb.rbody + w.delta;
    const T inb = c_div(T(1), T(rb.nb));
    T lsum = T(0);
#pragma unroll
    for (int i = 0; i < N; ++i) lsum += ch.L[i];
    const T marg = T(1e-4) * (lsum + gap);
    T mid[N][3];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      T q[3], s, c;
      backbone_point(ch.Rb[i], ch.pb[i], ch.ax[i], ch.ay[i], ch.x[i], ch.L[i], T(0.5), q, mid[i], s, c);
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
      for (int j = i + 2; j < N; ++j) {
        {
          const T dx = mid[i][0] - mid[j][0], dy = mid[i][1] - mid[j][1], dz = mid[i][2] - mid[j][2];
          const T lim = T(0.5) * (ch.L[i] + ch.L[j]) + gap + marg;
          if (!(dx * dx + dy * dy + dz * dz < lim * lim)) continue;
        }
        const T limj = T(0.5) * ch.L[j] + gap + marg;
        for (int ka = 1; ka <= rb.nb; ++ka) {
          const T sa = T(ka) * inb;
          T qa[3], pa[3], s_a, c_a;
          backbone_point(ch.Rb[i], ch.pb[i], ch.ax[i], ch.ay[i], ch.x[i], ch.L[i], sa, qa, pa, s_a, c_a);
          {
            const T ex = pa[0] - mid[j][0], ey = pa[1] - mid[j][1], ez = pa[2] - mid[j][2];
            if (!(ex * ex + ey * ey + ez * ez < limj * limj)) continue;
          }
          for (int kb = 1; kb <= rb.nb; ++kb) {
            const T sb = T(kb) * inb;
            T qb[3], pb[3], s_b, c_b;
            backbone_point(ch.Rb[j], ch.pb[j], ch.ax[j], ch.ay[j], ch.x[j], ch.L[j], sb, qb, pb, s_b, c_b);
            const T dx = pa[0] - pb[0], dy = pa[1] - pb[1], dz = pa[2] - pb[2];
            const T d2 = dx * dx + dy * dy + dz * dz;
            if (!(d2 < gap * gap)) continue;
            const T dist = c_sqrt(d2);
            const T rr = w.ss * (gap - dist);
            F += T(0.5) * rr * rr;
            const T nh[3] = {dx / dist, dy / dist, dz / dist};
            T jr[D];
#pragma unroll
            for (int qq = 0; qq < D; ++qq) jr[qq] = T(0);
            add_sample_row<T, N, MODEL>(rb, ch, tv, tw, ldir, i, sa, qa, pa, s_a, c_a, nh, -w.ss, jr);
            add_sample_row<T, N, MODEL>(rb, ch, tv, tw, ldir, j, sb, qb, pb, s_b, c_b, nh, w.ss, jr);
            to_actuator<MODEL, T, N>(jr);
            rank1<TA, D>(A, g, jr, rr);
          }
        }
      }
    }
  }
  return F;
}

// ------------------------------------------------------------------------------------------------
// FP64 reciprocal for the pivots of the block solves
// ------------------------------------------------------------------------------------------------
// 1/d by Newton-Raphson iteration for the reciprocal, r <- r + r (1 - d r), started from the
// single-precision hardware approximation (PTX rcp.approx.f32, within 1 ulp of float). The seed's
// relative error e (<= 2^-22 with the rounding of d to float) becomes e^2 after one step and e^4
// after two, below FP64 rounding, so the result is within a few ulp of 1/d. Four FMAs on the FP64
// pipe instead of the longer division sequence. Outside the single-precision normal range the
// division is taken.
CR_HD double recip_nr(double d) {
  const double ad = d < 0.0 ? -d : d;
  if (!(ad > 1e-37 && ad < 1e37)) return 1.0 / d;
  const float f = __double2float_rn(d);
  float rf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(f));
  double r = double(rf);
  double e = fma(-d, r, 1.0);
  r = fma(r, e, r);
  e = fma(-d, r, 1.0);
  return fma(r, e, r);
}

// ------------------------------------------------------------------------------------------------
// FP64 Cholesky of a packed lower-triangular matrix and the two triangular solves.
// ------------------------------------------------------------------------------------------------
// The reciprocal pivots are kept in invd[] so that the solves multiply instead of divide (FP64
// division and square root are long instruction sequences on a part with a narrow FP64 pipe).
// Every loop has a constant trip count with the triangular range as a guard, so that full unrolling
// leaves only constant indices and the packed matrix stays in registers (with trip counts that depend
// on an outer index the compiler kept it in local memory).
template <int D> CR_HD bool cholesky_packed(double (&A)[D * (D + 1) / 2], double (&invd)[D]) {
  bool ok = true;  // no early exit: keeps the fully unrolled factorisation in registers
#pragma unroll
  for (int j = 0; j < D; ++j) {
    double s = A[tri(j, j)];
#pragma unroll
    for (int k = 0; k < D; ++k)
      if (k < j) s -= A[tri(j, k)] * A[tri(j, k)];
    ok = ok && (s > 0.0);
    s = s > 0.0 ? s : 1.0;
    double inv = rsqrt(s);
    double ljj = s * inv;
    invd[j] = inv;
    A[tri(j, j)] = ljj;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      if (i <= j) continue;
      double t = A[tri(i, j)];
#pragma unroll
      for (int k = 0; k < D; ++k)
        if (k < j) t -= A[tri(i, k)] * A[tri(j, k)];
      A[tri(i, j)] = t * inv;
    }
  }
  return ok;
}

template <int D>
CR_HD void cholesky_solve(const double (&Lm)[D * (D + 1) / 2], const double (&invd)[D], double (&x)[D]) {
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double s = x[i];
#pragma unroll
    for (int k = 0; k < D; ++k)
      if (k < i) s -= Lm[tri(i, k)] * x[k];
    x[i] = s * invd[i];
  }
#pragma unroll
  for (int i = D - 1; i >= 0; --i) {
    double s = x[i];
#pragma unroll
    for (int k = 0; k < D; ++k)
      if (k > i) s -= Lm[tri(k, i)] * x[k];
    x[i] = s * invd[i];
  }
}

// ------------------------------------------------------------------------------------------------
// Projection of one segment onto {|u_j| <= b, sum u_j = 0}: u_j = clamp(v_j - tau, -b, b), with
// tau the root of g(tau) = sum_j clamp(v_j - tau, -b, b); g is non-increasing and piecewise linear
// with breakpoints v_j -/+ b, so tau lies between the largest breakpoint with g >= 0 and the
// smallest with g <= 0 and follows by linear interpolation.
// ------------------------------------------------------------------------------------------------
template <typename T> CR_HD void project3(T v0, T v1, T v2, T b, T& u0, T& u1, T& u2) {
  // interior: the projection onto the plane sum u = 0 already satisfies the bounds (tau = mean)
  T m = (v0 + v1 + v2) * T(1.0 / 3.0);
  T w0 = v0 - m, w1 = v1 - m, w2 = v2 - m;
  if (c_fabs(w0) <= b && c_fabs(w1) <= b && c_fabs(w2) <= b) {
    u0 = w0; u1 = w1; u2 = w2;
    return;
  }
  // Otherwise, with va >= vb >= vc the solution has u_a >= 0 >= u_c and u_b strictly inside, so
  // only u_a can clamp (at +b) and only u_c (at -b): g(tau) = min(va - tau, b) + (vb - tau) +
  // max(vc - tau, -b). Its breakpoints are va - b and vc + b; the sign of g at them selects which
  // of the four linear pieces holds the root, and each piece has a closed-form root.
  T va = c_max(v0, c_max(v1, v2)), vc = c_min(v0, c_min(v1, v2));
  T vb = c_max(c_min(v0, v1), c_min(c_max(v0, v1), v2));  // median
  T tT = va - b, tB = vc + b;
  T lo = c_min(tT, tB), hi = c_max(tT, tB);
  T glo = c_min(va - lo, b) + (vb - lo) + c_max(vc - lo, -b);
  T ghi = c_min(va - hi, b) + (vb - hi) + c_max(vc - hi, -b);
  T t_top = T(0.5) * (vb + vc + b);   // u_a = b
  T t_bot = T(0.5) * (va + vb - b);   // u_c = -b
  T t_mid = tT <= tB ? m : vb;        // no clamp, or both (u_b = 0)
  T tau = glo < T(0) ? t_top : (ghi > T(0) ? t_bot : t_mid);
  u0 = clampb(v0 - tau, b);
  u1 = clampb(v1 - tau, b);
  u2 = clampb(v2 - tau, b);
}

// Arc model: projection onto {theta <= theta_max} x [l_min, l_max] (a disk times an interval, each
// factor on its own): the bend scaled back radially onto the disk, the length clamped.
template <typename T>
CR_HD void project_arc(T v0, T v1, T v2, T thmax, T lmin, T lmax, T& u0, T& u1, T& u2) {
  const T r2 = v0 * v0 + v1 * v1;
  const T f = r2 > thmax * thmax ? thmax / c_sqrt(r2) : T(1);
  u0 = v0 * f;
  u1 = v1 * f;
  u2 = c_min(lmax, c_max(lmin, v2));
}

template <int MODEL, typename T, int N>
CR_HD void project_state(const RobotK<T>& rb, const T (&v)[3 * N], T (&u)[3 * N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if (MODEL == CR_MODEL_ARC)
      project_arc(v[3 * i], v[3 * i + 1], v[3 * i + 2], rb.thmax[i], rb.lmin[i], rb.lmax[i], u[3 * i], u[3 * i + 1],
                  u[3 * i + 2]);
    else
      project3(v[3 * i], v[3 * i + 1], v[3 * i + 2], rb.umax[i], u[3 * i], u[3 * i + 1], u[3 * i + 2]);
  }
}

// ------------------------------------------------------------------------------------------------
// Counter-based seeds: SplitMix64 (Steele, Lea, Flood 2014), output k from state s0 is
// mix(s0 + k * 0x9E3779B97F4A7C15). A seed is uniform on each segment's hexagon: rhombus
// k = floor(3 U0), then U1 V_2k + U2 V_2k+2 with V the hexagon vertices in cyclic order.
// ------------------------------------------------------------------------------------------------
CR_HD uint64_t splitmix64_at(uint64_t s0, uint64_t k) {
  uint64_t z = s0 + k * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
CR_HD double u01(uint64_t z) { return (double)(z >> 11) * (1.0 / 9007199254740992.0); }
CR_HD uint64_t seed_counter(uint64_t p, uint64_t s, uint64_t a, uint64_t i, uint64_t w) {
  return ((((p * 65536ULL + s) * 8ULL + a) * 8ULL + i) * 4ULL + w) + 1ULL;
}

// Hexagon vertices in cyclic order, as signs of b: (b,0,-b), (b,-b,0), (0,-b,b), (-b,0,b), (-b,b,0), (0,b,-b).
CR_HD int hex_sign(int v, int j) {
  // table packed as 2-bit codes: 0 -> 0, 1 -> +1, 2 -> -1
  const int code[6] = {0x21, 0x09, 0x18, 0x12, 0x06, 0x24};  // bits (j=0: 1:0, j=1: 3:2, j=2: 5:4)
  int c = (code[v] >> (2 * j)) & 3;
  return c == 1 ? 1 : (c == 2 ? -1 : 0);
}

// FP64, IEEE round-to-nearest without contraction (bitwise-reproducible against a CPU double
// implementation of the same formula).
CR_HD void hexagon_point(double b, double U0, double U1, double U2, double (&u)[3]) {
  int k = (int)__dmul_rn(3.0, U0);
  if (k > 2) k = 2;
  int va = 2 * k, vb = (2 * k + 2) % 6;
  double ab = __dmul_rn(U1, b), bb = __dmul_rn(U2, b);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    int sa = hex_sign(va, j), sb = hex_sign(vb, j);
    double ta = sa == 0 ? 0.0 : (sa > 0 ? ab : -ab);
    double tb = sb == 0 ? 0.0 : (sb > 0 ? bb : -bb);
    u[j] = __dadd_rn(ta, tb);
  }
}

template <typename T, int N>
CR_HD void draw_seed(uint64_t key, uint64_t p, uint64_t s, int attempt, const double (&umax)[NMAX],
                     T (&u)[3 * N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    double U0 = u01(splitmix64_at(key, seed_counter(p, s, attempt, i, 0)));
    double U1 = u01(splitmix64_at(key, seed_counter(p, s, attempt, i, 1)));
    double U2 = u01(splitmix64_at(key, seed_counter(p, s, attempt, i, 2)));
    double uu[3];
    hexagon_point(umax[i], U0, U1, U2, uu);
    u[3 * i] = T(uu[0]);
    u[3 * i + 1] = T(uu[1]);
    u[3 * i + 2] = T(uu[2]);
  }
}

// Bounds of the seed draws, FP64: the tendon model's u_max, the arc model's theta_max and lengths.
struct SeedBox {
  double umax[NMAX], thmax[NMAX], lmin[NMAX], lmax[NMAX];
};

// Arc-model seed (see cr_model): L_i uniform on [l_min, l_max] (draw 0); the bend uniform on the disk
// of radius theta_max by rejection from the enclosing square, try t = 0..7 taking the square's point
// from draws 1 and 2 at counters offset by t 2^48 (beyond every draw counter of problems p < 2^24);
// if no try falls inside, the last is scaled onto the circle. FP64 with explicit roundings (no
// contraction), bitwise reproducible against a CPU double implementation of the same steps.
template <typename T, int N>
CR_HD void draw_seed_arc(uint64_t key, uint64_t p, uint64_t s, int attempt, const SeedBox& bx, T (&u)[3 * N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const double th = bx.thmax[i], th2 = __dmul_rn(th, th);
    const double UL = u01(splitmix64_at(key, seed_counter(p, s, attempt, i, 0)));
    double x = 0.0, y = 0.0;
    bool in = false;
    for (uint64_t t = 0; t < 8 && !in; ++t) {
      const double X = u01(splitmix64_at(key, seed_counter(p, s, attempt, i, 1) + (t << 48)));
      const double Y = u01(splitmix64_at(key, seed_counter(p, s, attempt, i, 2) + (t << 48)));
      x = __dmul_rn(__dsub_rn(__dmul_rn(2.0, X), 1.0), th);
      y = __dmul_rn(__dsub_rn(__dmul_rn(2.0, Y), 1.0), th);
      in = __dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)) <= th2;
    }
    if (!in) {
      const double f = __ddiv_rn(th, __dsqrt_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y))));
      x = __dmul_rn(x, f);
      y = __dmul_rn(y, f);
    }
    u[3 * i] = T(x);
    u[3 * i + 1] = T(y);
    u[3 * i + 2] = T(__dadd_rn(bx.lmin[i], __dmul_rn(UL, __dsub_rn(bx.lmax[i], bx.lmin[i]))));
  }
}

inline SeedBox seed_box(const cr_robot& r) {
  SeedBox b;
  for (int i = 0; i < NMAX; ++i) {
    const bool on = i < r.n;
    b.umax[i] = on ? r.u_max[i] : 0.0;
    b.thmax[i] = on ? r.theta_max[i] : 0.0;
    b.lmin[i] = on && r.model == CR_MODEL_ARC ? r.l_min[i] : 0.0;
    b.lmax[i] = on && r.model == CR_MODEL_ARC ? r.l_max[i] : 0.0;
  }
  return b;
}

template <int MODEL, typename T, int N>
CR_HD void draw_seed_m(uint64_t key, uint64_t p, uint64_t s, int attempt, const SeedBox& bx, T (&u)[3 * N]) {
  if (MODEL == CR_MODEL_ARC) draw_seed_arc<T, N>(key, p, s, attempt, bx, u);
  else draw_seed<T, N>(key, p, s, attempt, bx.umax, u);
}

// Does any backbone sample of state u come within reach of an obstacle?
template <typename T, int N, int MODEL = CR_MODEL_TENDON>
CR_HD bool state_collides(const RobotK<T>& rb, ObsK<T> ob, int no, const T (&u)[3 * N]) {
  const Sphere4<T>* sph = ob.s;
  Chain<T, N> ch;
  chain_forward<T, N, MODEL>(rb, u, ch);
  const T inb = T(1) / T(rb.nb);
  for (int j0 = 0; j0 < no; j0 += 64) {
    uint64_t mk[N];
    segment_sphere_masks(rb, ch, ob, j0, no - j0 < 64 ? no - j0 : 64, mk);
    for (int i = 0; i < N; ++i) {
      if (!mk[i]) continue;
      for (int k0 = 1; k0 <= rb.nb; k0 += kCullGroup) {
      const int k1 = k0 + kCullGroup - 1 < rb.nb ? k0 + kCullGroup - 1 : rb.nb;
      const uint64_t gm = group_sphere_mask<T, N>(rb, ch, i, k0, k1, ob, j0, mk[i]);
      if (!gm) continue;
      for (int k = k0; k <= k1; ++k) {
        T q[3], wp[3], s, c;
        backbone_point(ch.Rb[i], ch.pb[i], ch.ax[i], ch.ay[i], ch.x[i], ch.L[i], T(k) * inb, q, wp, s, c);
        const uint64_t sb = sphere_bits(ob, j0);
        for (uint64_t bits = gm & sb; bits; bits &= bits - 1) {
          Sphere4<T> S = sph[j0 + __ffsll((long long)bits) - 1];
          T dx = wp[0] - S.x, dy = wp[1] - S.y, dz = wp[2] - S.z;
          if (dx * dx + dy * dy + dz * dz < S.reach * S.reach) return true;
        }
        for (uint64_t bits = ob.prims() ? gm & ~sb : 0ull; bits; bits &= bits - 1) {
          const PrimK<T>& P = ob.p[j0 + __ffsll((long long)bits) - 1 - ob.ns];
          T viol, nv[3];
          if (prim_active(P, wp, P.reach, viol, nv)) return true;
        }
      }
      }
    }
  }
  return false;
}

}  // namespace crk
