// FP64 CPU oracle of the CR-Solver hot path (tendon-driven continuum robots).
//
// TEST INFRASTRUCTURE ONLY. This is the plain, slow, obviously-correct reference that the CUDA
// library is checked against. It shares no code, header, table or helper with the CUDA path and
// never includes any of its files. Only the test-suite, the smoke check and the CPU-baseline leg
// of the benchmark load it. Product code must never call into it.
//
// What it computes, in the paper's order and notation:
//   * Sec. III-A, Eq. 1-3: segment transform T_{i-1}^i = [R d; 0 1] with R = Z(phi) Y(theta) Z(-phi)
//     and d = r [cos phi (1-cos theta), sin phi (1-cos theta), sin theta], r = L/theta, d = [0,0,L]
//     at theta = 0 (written as its Taylor expansion about the straight configuration there).
//   * Sec. III-B, Eq. 4: tendon length l_ij = L_i - r_c theta_i cos(alpha_j - phi_i), read per segment
//     (each segment carries its own m tendons); the decision variable is the displacement
//     u_ij = l_ij - L_i, and (theta_i, phi_i) follow from u_i by the exact inverse of Eq. 4.
//   * Sec. IV-A: IK objective ||log(T_ee^-1 T_target)|| (Eq. ik_opt) read as the split residual
//     [w_p (p_ee - p_t); w_R Log(R_t^T R_ee)], bound constraint (Eq. ik_limits), clearance
//     constraint (Eq. ik_coll), trajectory objective and tendon velocity/acceleration limits
//     (Eq. mp_length_only and the finite differences after it), path-following objective
//     (Eq. constrained_mp).
//   * Sec. IV-B, Eq. penalized_form: cost = f + rho_ineq Pi_ineq(c) + rho_eq Pi_eq(h) written as a
//     least-squares sum 1/2 sum r^2 (Sec. VI calls it a penalised least-squares form) with
//     squared-hinge inequality rows and plain equality rows.
//   * Sec. IV-C: batched Levenberg-Marquardt with dense Cholesky (Marquardt diagonal scaling,
//     gain-ratio damping update of Madsen, Nielsen and Tingleff).
//   * Algorithm 1 (beam search IK): SampleSeeds -> ParallelOptimize(k_init) -> SelectTop(N_final) ->
//     ParallelOptimize(k_final) -> argmin.
//   * Trajectory planning (Sec. IV-A, Eq. mp_length_only with the tendon speed / acceleration
//     limits by finite differences; Alg. 2's refinement stage after the linear initialiser of
//     Sec. V-C): goal IK, linear interpolation, projected-gradient refinement of all states.
//   * Path following (Sec. IV-A, Eq. constrained_mp; Sec. IV-B "Path Following"): IK at the first
//     waypoint, warm-started per-waypoint IK, then joint LM over all waypoints with successive-state
//     smoothness rows and a dense Cholesky of the whole normal matrix.
//   * Kinematic calibration of segment lengths and tendon radii from measured tip positions (LM).
//   * PRM exploration of Algorithm 2: ParallelSample, ParallelConnect (k nearest neighbours and
//     collision-checked straight edges), ConnectToRoadmap, Dijkstra and ResampleLinear.
//   * Self-contact rows between backbone samples of non-adjacent segments (Eq. ik_coll over the
//     robot itself), as standalone functions.
//   * Obstacles as convex pieces (Sec. IV-C): spheres, capsules and boxes, each entering the
//     clearance rows through its signed distance.
//   * Coupled tendon routing (Eq. l_eq summed over the segments a tendon runs through): the map
//     between per-segment and actuator displacements, as standalone functions.
//
// Derivatives are taken by the complex-step method (Squire and Trapp 1998): for a real-analytic
// function f, f'(x) = Im f(x + i h) / h up to O(h^2), with no subtractive cancellation, so with
// h = 1e-30 the Jacobian is exact to rounding. Every function below is templated on its scalar so
// that the same code runs on double, on std::complex<double> (for derivatives), and on an
// op-counting scalar (for the algorithmic flop counts the benchmark divides by).
//
// Build: g++ -std=c++17 -O2 -fPIC -shared -ffp-contract=off -pthread (no -ffast-math, no SIMD
// intrinsics; -ffp-contract=off keeps x86-64 and aarch64 results identical).

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <functional>
#include <queue>
#include <thread>
#include <vector>

typedef std::complex<double> cd;

// ---------------------------------------------------------------------------------------------
// Scalars: double, complex (complex step), and an op-counting scalar.
// ---------------------------------------------------------------------------------------------

// Op tally for algorithmic counts: forward ("value") flops and special-function calls, and the
// flops / special calls of the linearised program (the tangent map, which the adjoint transposes
// with the same number of multiply-adds). Single-threaded use only.
struct OpTally {
  long long f_flop, f_sfu, t_flop, t_sfu;
};
static OpTally g_tally = {0, 0, 0, 0};

struct Cnt {
  double v;  // value
  bool a;    // depends on the differentiated input (tangent structurally non-zero)
  Cnt() : v(0), a(false) {}
  Cnt(double x) : v(x), a(false) {}
  Cnt(double x, bool act) : v(x), a(act) {}
};
static inline Cnt operator+(Cnt x, Cnt y) {
  g_tally.f_flop++;
  if (x.a && y.a) g_tally.t_flop++;
  return Cnt(x.v + y.v, x.a || y.a);
}
static inline Cnt operator-(Cnt x, Cnt y) {
  g_tally.f_flop++;
  if (x.a && y.a) g_tally.t_flop++;
  return Cnt(x.v - y.v, x.a || y.a);
}
static inline Cnt operator-(Cnt x) { return Cnt(-x.v, x.a); }
static inline Cnt operator*(Cnt x, Cnt y) {
  g_tally.f_flop++;
  if (x.a && y.a) g_tally.t_flop += 3;
  else if (x.a || y.a) g_tally.t_flop += 1;
  return Cnt(x.v * y.v, x.a || y.a);
}
static inline Cnt operator/(Cnt x, Cnt y) {
  g_tally.f_flop++;
  if (y.a) g_tally.t_flop += x.a ? 3 : 2;
  else if (x.a) g_tally.t_flop += 1;
  return Cnt(x.v / y.v, x.a || y.a);
}
static inline Cnt& operator+=(Cnt& x, Cnt y) { x = x + y; return x; }
static inline Cnt& operator-=(Cnt& x, Cnt y) { x = x - y; return x; }
static inline Cnt& operator*=(Cnt& x, Cnt y) { x = x * y; return x; }

static inline double re(double x) { return x; }
static inline double re(const cd& x) { return x.real(); }
static inline double re(const Cnt& x) { return x.v; }

static inline double Sqrt(double x) { return std::sqrt(x); }
static inline cd Sqrt(const cd& x) { return std::sqrt(x); }
static inline Cnt Sqrt(Cnt x) {
  g_tally.f_sfu++;
  if (x.a) g_tally.t_flop += 2;
  return Cnt(std::sqrt(x.v), x.a);
}
static inline double Sin(double x) { return std::sin(x); }
static inline cd Sin(const cd& x) { return std::sin(x); }
static inline Cnt Sin(Cnt x) {
  g_tally.f_sfu++;
  if (x.a) { g_tally.t_sfu++; g_tally.t_flop++; }
  return Cnt(std::sin(x.v), x.a);
}
static inline double Cos(double x) { return std::cos(x); }
static inline cd Cos(const cd& x) { return std::cos(x); }
static inline Cnt Cos(Cnt x) {
  g_tally.f_sfu++;
  if (x.a) { g_tally.t_sfu++; g_tally.t_flop++; }
  return Cnt(std::cos(x.v), x.a);
}
static inline double Atan2(double y, double x) { return std::atan2(y, x); }
// atan2 is not complex-analytic as a library call; its complex-step extension only needs the
// first-order term: atan2(y, x) + i (x Im y - y Im x) / (x^2 + y^2), evaluated at the real parts.
static inline cd Atan2(const cd& y, const cd& x) {
  double xr = x.real(), yr = y.real();
  double den = xr * xr + yr * yr;
  double d = den > 0 ? (xr * y.imag() - yr * x.imag()) / den : 0.0;
  return cd(std::atan2(yr, xr), d);
}
static inline Cnt Atan2(Cnt y, Cnt x) {
  g_tally.f_sfu++;
  if (x.a || y.a) g_tally.t_flop += 6;
  return Cnt(std::atan2(y.v, x.v), x.a || y.a);
}

// Squared-hinge helper: max(0, x), decided on the real part (derivative 0 at exactly 0).
template <class T> static inline T hinge(const T& x) { return re(x) > 0.0 ? x : T(0.0); }

// ---------------------------------------------------------------------------------------------
// Parameters (plain C structs, mirrored by ctypes in oracle/__init__.py)
// ---------------------------------------------------------------------------------------------

#define OR_MAXSEG 8

struct OrRobot {
  int32_t n;   // segments
  int32_t m;   // tendons per segment (equally spaced, alpha_j = (j-1) 2 pi / m)
  int32_t nb;  // backbone samples per segment (sample k at arc fraction k/nb, k = 1..nb)
  int32_t model;  // decision variables: OR_MODEL_TENDON or OR_MODEL_ARC (see below)
  double L[OR_MAXSEG];      // segment arc length (m)
  double rc[OR_MAXSEG];     // tendon routing radius (m)
  double umax[OR_MAXSEG];   // displacement bound |u_ij| <= umax_i (m)
  double thmax[OR_MAXSEG];  // bending-angle limit (rad)
  double rbody;             // backbone radius used by the clearance rows (m)
  double lmin[OR_MAXSEG];   // OR_MODEL_ARC: arc-length bounds lmin_i <= L_i <= lmax_i (m)
  double lmax[OR_MAXSEG];
};

// Decision variables of a segment. OR_MODEL_TENDON: the m tendon displacements u_ij (Eq. 4 gives
// theta, phi; L is the robot's). OR_MODEL_ARC: the paper's own configuration q_i = (theta, phi, L)
// of Sec. IV-A, with L free within [lmin, lmax] (extendable segments) and (theta, phi) written in
// Cartesian form (theta cos phi, theta sin phi): the same configurations, smooth at theta = 0 where
// phi is undefined. Three variables per segment in both models.
// OR_MODEL_COUPLED: coupled tendon routing (model B, Eq. l_eq read literally, reading 23): the tendons
// that end at segment s run through segments 1..s, and the state holds their actuator displacements
// q_sj = sum_{i <= s} u_ij; the kinematics take the per-segment displacements u_s = q_s - q_{s-1}
// (the inverse of the prefix sum); bounds |q_sj| <= umax_s and sum_j q_sj = 0 act on the actuators.
enum { OR_MODEL_TENDON = 0, OR_MODEL_ARC = 1, OR_MODEL_COUPLED = 2 };
#define OR_MAXM 16

struct OrWeights {
  double wp, wR;                         // pose residual weights (1/m, 1/rad)
  double rho_b, rho_eq, rho_k, rho_c;    // penalty weights: bounds, sum-zero, curvature, clearance
  double w_s, w_len, rho_v, rho_a;       // path smoothness, path length, tendon vel / acc
  double dt, vmax, amax;                 // time step, tendon speed / acceleration limits
  double delta;                          // safety margin of Eq. ik_coll (m)
  double rho_s;                          // self-contact rows (reading: pairs of segments two or more
                                         // apart); 0 leaves them out
};

enum { OR_IK6 = 0, OR_IK5 = 1 };

// ---------------------------------------------------------------------------------------------
// Kinematics (Sec. III)
// ---------------------------------------------------------------------------------------------

// Exact inverse of Eq. 4 for one segment. With u_j = l_j - L = -r_c theta cos(alpha_j - phi) and m
// >= 3 equally spaced tendons, sum_j cos(alpha_j - phi) cos(alpha_j) = (m/2) cos(phi) and
// sum_j cos(alpha_j - phi) sin(alpha_j) = (m/2) sin(phi). Returns tx = theta cos phi and
// ty = theta sin phi.
template <class T>
static void tendon_to_bend(const T* u, int m, const T& rc, T& tx, T& ty) {
  T sx(0.0), sy(0.0);
  for (int j = 0; j < m; ++j) {
    double alpha = 2.0 * M_PI * j / m;
    sx += u[j] * T(std::cos(alpha));
    sy += u[j] * T(std::sin(alpha));
  }
  T k = T(-2.0 / m) / rc;
  tx = k * sx;
  ty = k * sy;
}

// Eq. 4 forward: displacement of tendon j for a segment bent by (theta, phi).
static double tendon_displacement(double rc, double theta, double phi, int j, int m) {
  double alpha = 2.0 * M_PI * j / m;
  return -rc * theta * std::cos(alpha - phi);
}

template <class T> static void rot_z(const T& a, T M[3][3]) {
  T c = Cos(a), s = Sin(a);
  M[0][0] = c;      M[0][1] = -s;     M[0][2] = T(0.0);
  M[1][0] = s;      M[1][1] = c;      M[1][2] = T(0.0);
  M[2][0] = T(0.0); M[2][1] = T(0.0); M[2][2] = T(1.0);
}
template <class T> static void rot_y(const T& a, T M[3][3]) {
  T c = Cos(a), s = Sin(a);
  M[0][0] = c;      M[0][1] = T(0.0); M[0][2] = s;
  M[1][0] = T(0.0); M[1][1] = T(1.0); M[1][2] = T(0.0);
  M[2][0] = -s;     M[2][1] = T(0.0); M[2][2] = c;
}
template <class T> static void matmul3(const T A[3][3], const T B[3][3], T C[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T s = A[i][0] * B[0][j];
      s += A[i][1] * B[1][j];
      s += A[i][2] * B[2][j];
      C[i][j] = s;
    }
}

// Below this theta^2 the segment uses the Taylor expansion of Eq. 2-3 about theta = 0 (the paper
// only states d = [0,0,L] at theta = 0; phi is undefined there).
static const double OR_SMALL_TH2 = 1e-8;

// Rodrigues / series form of Eq. 2-3 in terms of (tx, ty) = theta (cos phi, sin phi):
// R = I + s [w]x + c [w]x^2 with w = (-ty, tx, 0), s = sin(theta)/theta, c = (1-cos theta)/theta^2,
// d = L (c tx, c ty, s). Identical to the ZYZ product; used for small theta (with the series of s
// and c) and, with exact s and c, by the op counter as the minimal arithmetic form of Eq. 2-3.
template <class T>
static void segment_rodrigues(const T& tx, const T& ty, const T& L, const T& s, const T& c,
                              T R[3][3], T d[3]) {
  T cxy = c * tx * ty;
  R[0][0] = T(1.0) - c * tx * tx; R[0][1] = -cxy;                 R[0][2] = s * tx;
  R[1][0] = -cxy;                 R[1][1] = T(1.0) - c * ty * ty; R[1][2] = s * ty;
  R[2][0] = -(s * tx);            R[2][1] = -(s * ty);            R[2][2] = T(1.0) - c * (tx * tx + ty * ty);
  d[0] = L * c * tx;
  d[1] = L * c * ty;
  d[2] = L * s;
}

static bool g_count_minimal = false;  // op counting: use the minimal (Rodrigues) arithmetic form
// op counting: leave out the rows that vanish on the feasible set of stage one's projection (the form
// a projected trial point is evaluated in): the tendon model's bound and sum-zero rows, the arc
// model's length and curvature rows
static bool g_count_skip_box = false;

// Segment transform T_{i-1}^i of Eq. 1: rotation R (Eq. 2) and translation d (Eq. 3).
template <class T>
static void segment_transform(const T& tx, const T& ty, const T& L, T R[3][3], T d[3]) {
  T th2 = tx * tx + ty * ty;
  if (re(th2) < OR_SMALL_TH2) {
    // Taylor series of sin(theta)/theta and (1-cos theta)/theta^2 in theta^2.
    T s = T(1.0) - th2 / T(6.0) + th2 * th2 / T(120.0);
    T c = T(0.5) - th2 / T(24.0) + th2 * th2 / T(720.0);
    segment_rodrigues(tx, ty, L, s, c, R, d);
    return;
  }
  T th = Sqrt(th2);
  if (g_count_minimal) {
    T h = th / T(2.0);
    T sh = Sin(h), ch = Cos(h);
    T sc = sh / h;
    T s = sc * ch, c = T(0.5) * sc * sc;
    segment_rodrigues(tx, ty, L, s, c, R, d);
    return;
  }
  T phi = Atan2(ty, tx);
  // Eq. 2: R = Z(phi) Y(theta) Z(-phi)
  T Zp[3][3], Y[3][3], Zm[3][3], ZY[3][3];
  rot_z(phi, Zp);
  rot_y(th, Y);
  rot_z(-phi, Zm);
  matmul3(Zp, Y, ZY);
  matmul3(ZY, Zm, R);
  // Eq. 3 with r = L/theta; 1 - cos(theta) written as 2 sin^2(theta/2) (same value, no cancellation).
  T r = L / th;
  T sh = Sin(th / T(2.0));
  T omc = T(2.0) * sh * sh;
  d[0] = r * Cos(phi) * omc;
  d[1] = r * Sin(phi) * omc;
  d[2] = r * Sin(th);
}

// Per-segment kinematic parameters in scalar T (so that L and r_c can be differentiated).
template <class T> struct Params {
  T L[OR_MAXSEG];
  T rc[OR_MAXSEG];
};
template <class T> static Params<T> params_of(const OrRobot& rb) {
  Params<T> P;
  for (int i = 0; i < rb.n; ++i) { P.L[i] = T(rb.L[i]); P.rc[i] = T(rb.rc[i]); }
  return P;
}

// Forward kinematics by chaining Eq. 1 (T_0^n = T_0^1 T_1^2 ... T_{n-1}^n). Optionally writes the
// base frame of every segment (Rb[i], pb[i] = frame i-1), the backbone samples and theta_i.
template <class T> struct FkOut {
  T R[3][3];
  T p[3];
  T Rb[OR_MAXSEG][3][3];
  T pb[OR_MAXSEG][3];
  T th2[OR_MAXSEG];
};

template <class T> struct NoDeduce { typedef T type; };

template <class T>
static void forward_kinematics(const OrRobot& rb, const Params<T>& P, const T* u, FkOut<T>& o,
                               typename NoDeduce<T>::type* backbone /* [n*nb][3] or null */) {
  T R[3][3] = {{T(1.0), T(0.0), T(0.0)}, {T(0.0), T(1.0), T(0.0)}, {T(0.0), T(0.0), T(1.0)}};
  T p[3] = {T(0.0), T(0.0), T(0.0)};
  for (int i = 0; i < rb.n; ++i) {
    for (int a = 0; a < 3; ++a) {
      o.pb[i][a] = p[a];
      for (int b = 0; b < 3; ++b) o.Rb[i][a][b] = R[a][b];
    }
    T tx, ty, Li;
    if (rb.model == OR_MODEL_ARC) {
      tx = u[3 * i];
      ty = u[3 * i + 1];
      Li = u[3 * i + 2];
    } else if (rb.model == OR_MODEL_COUPLED) {
      T ui[OR_MAXM];
      for (int j = 0; j < rb.m; ++j) ui[j] = i == 0 ? u[j] : u[rb.m * i + j] - u[rb.m * (i - 1) + j];
      tendon_to_bend(ui, rb.m, P.rc[i], tx, ty);
      Li = P.L[i];
    } else {
      tendon_to_bend(u + rb.m * i, rb.m, P.rc[i], tx, ty);
      Li = P.L[i];
    }
    o.th2[i] = tx * tx + ty * ty;
    if (backbone) {
      // Backbone sample k: the arc of fraction sigma = k/nb, i.e. bending sigma*theta in the same
      // plane phi over arc length sigma*L, placed in the segment's base frame.
      for (int k = 1; k <= rb.nb; ++k) {
        T sg = T((double)k / rb.nb);
        T Rs[3][3], ds[3];
        segment_transform(sg * tx, sg * ty, sg * Li, Rs, ds);
        T* q = backbone + 3 * (i * rb.nb + (k - 1));
        for (int a = 0; a < 3; ++a) {
          if (i == 0) {  // the base frame is the identity at the origin
            q[a] = ds[a];
            continue;
          }
          T s = p[a];
          for (int b = 0; b < 3; ++b) s += R[a][b] * ds[b];
          q[a] = s;
        }
      }
    }
    T Ri[3][3], di[3];
    segment_transform(tx, ty, Li, Ri, di);
    if (i == 0) {  // T_0 itself: composing with the identity base frame changes no value
      for (int a = 0; a < 3; ++a) {
        p[a] = di[a];
        for (int b = 0; b < 3; ++b) R[a][b] = Ri[a][b];
      }
      continue;
    }
    T pn[3], Rn[3][3];
    for (int a = 0; a < 3; ++a) {
      T s = p[a];
      for (int b = 0; b < 3; ++b) s += R[a][b] * di[b];
      pn[a] = s;
    }
    matmul3(R, Ri, Rn);
    for (int a = 0; a < 3; ++a) {
      p[a] = pn[a];
      for (int b = 0; b < 3; ++b) R[a][b] = Rn[a][b];
    }
  }
  for (int a = 0; a < 3; ++a) {
    o.p[a] = p[a];
    for (int b = 0; b < 3; ++b) o.R[a][b] = R[a][b];
  }
}

// ---------------------------------------------------------------------------------------------
// SO(3) logarithm and pose residual (Eq. ik_opt, Eq. error_eq)
// ---------------------------------------------------------------------------------------------

// Log: SO(3) -> so(3) as a 3-vector w = angle * axis, angle in [0, pi]. The angle is
// atan2(|v|, (tr E - 1)/2) with v = vee(E - E^T)/2 = sin(angle) axis. Near angle 0 the factor
// angle/sin(angle) = asin(s)/s is a series in s^2 = |v|^2 (no square root of a vanishing number).
// Near angle pi the axis comes from the symmetric part (E + E^T)/2 = cos I + (1 - cos) n n^T,
// with its sign chosen so that n . v >= 0 (Sola, Deray, Atchuthan 2018, Sec. on SO(3) log).
template <class T> static void so3_log(const T E[3][3], T w[3]) {
  T v[3] = {(E[2][1] - E[1][2]) / T(2.0), (E[0][2] - E[2][0]) / T(2.0), (E[1][0] - E[0][1]) / T(2.0)};
  T cs = (E[0][0] + E[1][1] + E[2][2] - T(1.0)) / T(2.0);
  T s2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  if (re(cs) > 0.0 && re(s2) < 1e-6) {
    // asin(s)/s = 1 + s^2/6 + 3 s^4/40 + 5 s^6/112
    T f = T(1.0) + s2 / T(6.0) + T(3.0) * s2 * s2 / T(40.0) + T(5.0) * s2 * s2 * s2 / T(112.0);
    for (int a = 0; a < 3; ++a) w[a] = f * v[a];
    return;
  }
  if (re(cs) < 0.0 && re(s2) < 1e-2) {
    // near pi: n n^T = (S - cs I)/(1 - cs); take the column with the largest diagonal.
    T S[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) S[a][b] = (E[a][b] + E[b][a]) / T(2.0);
    int k = 0;
    for (int a = 1; a < 3; ++a)
      if (re(S[a][a]) > re(S[k][k])) k = a;
    T den = T(1.0) - cs;
    T nn_kk = (S[k][k] - cs) / den;
    T nk = Sqrt(nn_kk);
    T n[3];
    for (int a = 0; a < 3; ++a) n[a] = (a == k) ? nk : (S[a][k] / den) / nk;
    double dot = re(n[0]) * re(v[0]) + re(n[1]) * re(v[1]) + re(n[2]) * re(v[2]);
    T sgn = T(dot < 0.0 ? -1.0 : 1.0);
    T ang = Atan2(Sqrt(s2), cs);
    for (int a = 0; a < 3; ++a) w[a] = sgn * ang * n[a];
    return;
  }
  T sn = Sqrt(s2);
  T ang = Atan2(sn, cs);
  T f = ang / sn;
  for (int a = 0; a < 3; ++a) w[a] = f * v[a];
}

// Unit quaternion (w, x, y, z) -> rotation matrix (Hamilton convention).
static void quat_to_R(const double* q, double R[3][3]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  double nrm = std::sqrt(w * w + x * x + y * y + z * z);
  w /= nrm; x /= nrm; y /= nrm; z /= nrm;
  R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
  R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
  R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

// ---------------------------------------------------------------------------------------------
// Obstacles of the clearance rows (Eq. ik_coll). Sec. IV-C approximates a non-convex obstacle by a
// union of convex pieces; the pieces here are spheres, capsules and boxes. Each obstacle is a record
// of OR_OBS doubles: [0] kind, [1] radius r, then the kind's parameters. The clearance of a point x
// is its signed distance sd(x) to the obstacle's core set, less r:
//   kind 0, sphere:  core = the centre c = [2..4]; sd = |x - c|.
//   kind 1, capsule: core = the segment from a = [2..4] to b = [5..7]; sd = the distance from x to
//                    its nearest point a + t (b - a), t in [0, 1] (t = 0 when a = b).
//   kind 2, box:     core = the solid box with centre c = [2..4], half extents h = [5..7] and
//                    orientation the quaternion (w, x, y, z) = [8..11] (box frame to world, taken
//                    normalised). In box coordinates p = R^T (x - c), with q_a = |p_a| - h_a:
//                    outside (some q_a > 0) sd = the Euclidean distance to the box,
//                    sqrt(sum_a max(q_a, 0)^2); inside, sd = max_a q_a <= 0, minus the distance to
//                    the nearest face. With r > 0 the obstacle is a box with rounded edges.
// Any other kind reads as a sphere. A state's rows are sqrt(rho_c) max(0, r + r_body + delta - sd(p))
// over its backbone samples p and the obstacles.
static const int OR_OBS = 16;

static inline int obstacle_kind(const double* ob) {
  const int k = (int)ob[0];
  return k == 1 || k == 2 ? k : 0;
}

template <class T> static T obstacle_sd(const double* ob, const T* x) {
  const int kind = obstacle_kind(ob);
  if (kind == 1) {
    const double e[3] = {ob[5] - ob[2], ob[6] - ob[3], ob[7] - ob[4]};
    const double ee = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
    const T w[3] = {x[0] - T(ob[2]), x[1] - T(ob[3]), x[2] - T(ob[4])};
    T t(0.0);
    if (ee > 0.0) t = (w[0] * T(e[0]) + w[1] * T(e[1]) + w[2] * T(e[2])) / T(ee);
    if (re(t) < 0.0) t = T(0.0);
    if (re(t) > 1.0) t = T(1.0);
    const T d[3] = {w[0] - t * T(e[0]), w[1] - t * T(e[1]), w[2] - t * T(e[2])};
    return Sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  }
  if (kind == 2) {
    double R[3][3];
    quat_to_R(ob + 8, R);
    const T w[3] = {x[0] - T(ob[2]), x[1] - T(ob[3]), x[2] - T(ob[4])};
    T q[3];
    bool outside = false;
    for (int a = 0; a < 3; ++a) {
      T p = T(R[0][a]) * w[0] + T(R[1][a]) * w[1] + T(R[2][a]) * w[2];
      if (re(p) < 0.0) p = T(0.0) - p;
      q[a] = p - T(ob[5 + a]);
      if (re(q[a]) > 0.0) outside = true;
    }
    if (outside) {
      T s(0.0);
      for (int a = 0; a < 3; ++a)
        if (re(q[a]) > 0.0) s = s + q[a] * q[a];
      return Sqrt(s);
    }
    T m = q[0];
    for (int a = 1; a < 3; ++a)
      if (re(q[a]) > re(m)) m = q[a];
    return m;
  }
  const T d[3] = {x[0] - T(ob[2]), x[1] - T(ob[3]), x[2] - T(ob[4])};
  return Sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
}

// Is x closer than `reach` to the core of obstacle ob? On true, sd = its signed distance. Spheres
// decide on the squared distance, so that no square root is taken for an inactive pair.
template <class T> static bool obstacle_within(const double* ob, const T* x, double reach, T& sd) {
  if (obstacle_kind(ob) == 0) {
    const T dx = x[0] - T(ob[2]), dy = x[1] - T(ob[3]), dz = x[2] - T(ob[4]);
    const T d2 = dx * dx + dy * dy + dz * dz;
    if (!(re(d2) < reach * reach)) return false;
    sd = Sqrt(d2);
    return true;
  }
  sd = obstacle_sd(ob, x);
  return re(sd) < reach;
}

// Pose residual rows (6): IK6 -> [w_p (p - p_t); w_R Log(R_t^T R)]; IK5 -> [w_p (p - p_t); w_R (z - z_t)]
// where z is the tip axis (third column of R) and z_t the target axis.
template <class T>
static void pose_residual(int kind, const OrWeights& W, const double* tgt, const T R[3][3],
                          const T p[3], T* r) {
  for (int a = 0; a < 3; ++a) r[a] = T(W.wp) * (p[a] - T(tgt[a]));
  if (kind == OR_IK5) {
    double zn = std::sqrt(tgt[3] * tgt[3] + tgt[4] * tgt[4] + tgt[5] * tgt[5]);
    for (int a = 0; a < 3; ++a) r[3 + a] = T(W.wR) * (R[a][2] - T(tgt[3 + a] / zn));
    return;
  }
  double Rt[3][3];
  quat_to_R(tgt + 3, Rt);
  T E[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      T s = T(Rt[0][a]) * R[0][b];
      s += T(Rt[1][a]) * R[1][b];
      s += T(Rt[2][a]) * R[2][b];
      E[a][b] = s;
    }
  T w[3];
  so3_log(E, w);
  for (int a = 0; a < 3; ++a) r[3 + a] = T(W.wR) * w[a];
}

// ---------------------------------------------------------------------------------------------
// Constraint rows (Eq. ik_limits, ik_coll; Eq. penalized_form with squared hinges)
// ---------------------------------------------------------------------------------------------

// Self-contact rows (the robot itself in Eq. ik_coll's minimum distance, Sec. IV-A). Reading:
// backbone samples a of segment i and b of segment j >= i + 2 (adjacent segments meet at a joint,
// so their samples near it are always closer than any clearance), row
// sqrt(rho_s) max(0, 2 r_body + delta - |p_a - p_b|); rows in the order i, sample of i, j, sample of
// j. bb: the backbone samples [n*nb][3].
static int self_row_count(const OrRobot& rb) {
  int c = 0;
  for (int i = 0; i < rb.n; ++i)
    for (int j = i + 2; j < rb.n; ++j) c += rb.nb * rb.nb;
  return c;
}

template <class T>
static int self_rows_bb(const OrRobot& rb, const T* bb, double rho_s, double delta, T* r, T* pen) {
  const double gap = 2.0 * rb.rbody + delta;
  const T s = T(std::sqrt(rho_s));
  int k = 0;
  for (int i = 0; i < rb.n; ++i)
    for (int ka = 0; ka < rb.nb; ++ka)
      for (int j = i + 2; j < rb.n; ++j)
        for (int kb = 0; kb < rb.nb; ++kb) {
          const T* pa = bb + 3 * (i * rb.nb + ka);
          const T* pb = bb + 3 * (j * rb.nb + kb);
          T dx = pa[0] - pb[0], dy = pa[1] - pb[1], dz = pa[2] - pb[2];
          T d2 = dx * dx + dy * dy + dz * dz;
          if (re(d2) < gap * gap) {
            const T row = s * (T(gap) - Sqrt(d2));
            r[k++] = row;
            if (pen) *pen += row * row;
          } else {
            r[k++] = T(0.0);
          }
        }
  return k;
}

// Per-state constraint rows, appended at r; returns the number of rows.
// OR_MODEL_TENDON:
//   2d rows  sqrt(rho_b) max(0, u_ij - umax_i), sqrt(rho_b) max(0, -umax_i - u_ij)
//   n rows   sqrt(rho_eq) sum_j u_ij                      (common mode is invisible to FK)
// OR_MODEL_ARC (Eq. ik_limits on q = (theta, phi, L)):
//   2n rows  sqrt(rho_b) max(0, L_i - lmax_i), sqrt(rho_b) max(0, lmin_i - L_i)
// both:
//   n rows   sqrt(rho_k) max(0, theta_i - thmax_i)
//   n*nb*no  sqrt(rho_c) max(0, r_o + r_body + delta - sd_o(p_ik))   (sample-obstacle pairs)
template <class T>
static int state_constraint_rows(const OrRobot& rb, const OrWeights& W, int no,
                                 const double* obs, const T* u, const FkOut<T>& fk,
                                 const T* backbone, T* r, T* coll_pen) {
  int k = 0;
  const int d = rb.n * rb.m;
  T sb = T(std::sqrt(W.rho_b)), se = T(std::sqrt(W.rho_eq)), sk = T(std::sqrt(W.rho_k)),
    sc = T(std::sqrt(W.rho_c));
  if (rb.model == OR_MODEL_ARC) {
    for (int i = 0; i < rb.n && !g_count_skip_box; ++i) {
      r[k++] = sb * hinge(u[3 * i + 2] - T(rb.lmax[i]));
      r[k++] = sb * hinge(T(rb.lmin[i]) - u[3 * i + 2]);
    }
  } else if (!g_count_skip_box) {
    for (int q = 0; q < d; ++q) {
      int i = q / rb.m;
      r[k++] = sb * hinge(u[q] - T(rb.umax[i]));
      r[k++] = sb * hinge(T(-rb.umax[i]) - u[q]);
    }
    for (int i = 0; i < rb.n; ++i) {
      T s(0.0);
      for (int j = 0; j < rb.m; ++j) s += u[rb.m * i + j];
      r[k++] = se * s;
    }
  }
  // (the arc model's projected set holds theta <= theta_max, so its trial points need no curvature row)
  for (int i = 0; i < rb.n && !(g_count_skip_box && rb.model == OR_MODEL_ARC); ++i) {
    if (re(fk.th2[i]) > rb.thmax[i] * rb.thmax[i]) r[k++] = sk * (Sqrt(fk.th2[i]) - T(rb.thmax[i]));
    else r[k++] = T(0.0);
  }
  T cp(0.0);
  if (no > 0) {
    for (int q = 0; q < rb.n * rb.nb; ++q) {
      const T* x = backbone + 3 * q;
      for (int s = 0; s < no; ++s) {
        const double* ob = obs + OR_OBS * s;
        const double reach = ob[1] + rb.rbody + W.delta;
        T sd;
        if (obstacle_within(ob, x, reach, sd)) {
          T row = sc * (T(reach) - sd);
          r[k++] = row;
          cp += row * row;
        } else {
          r[k++] = T(0.0);
        }
      }
    }
  }
  // self-contact rows (their squares count as collision penalty too)
  if (W.rho_s > 0.0) k += self_rows_bb(rb, backbone, W.rho_s, W.delta, r + k, &cp);
  if (coll_pen) *coll_pen = cp;
  return k;
}

static int state_constraint_count(const OrRobot& rb, const OrWeights& W, int no) {
  const int self = W.rho_s > 0.0 ? self_row_count(rb) : 0;
  if (rb.model == OR_MODEL_ARC) return 3 * rb.n + rb.n * rb.nb * no + self;
  return 2 * rb.n * rb.m + 2 * rb.n + rb.n * rb.nb * no + self;
}

// Backbone samples are needed by the clearance rows and the self-contact rows.
static bool needs_backbone(const OrWeights& W, int no) { return no > 0 || W.rho_s > 0.0; }

// Full IK residual of one seed: 6 pose rows followed by the constraint rows.
template <class T>
static int ik_residual(const OrRobot& rb, const Params<T>& P, const OrWeights& W, int no,
                       const double* obs, int kind, const double* tgt, const T* u, T* r,
                       T* coll_pen) {
  FkOut<T> fk;
  const bool nbb = needs_backbone(W, no);
  std::vector<T> bb(nbb ? 3 * rb.n * rb.nb : 0);
  forward_kinematics(rb, P, u, fk, nbb ? bb.data() : nullptr);
  pose_residual(kind, W, tgt, fk.R, fk.p, r);
  return 6 + state_constraint_rows(rb, W, no, obs, u, fk, nbb ? bb.data() : nullptr, r + 6,
                                   coll_pen);
}

static int ik_rows(const OrRobot& rb, const OrWeights& W, int no) { return 6 + state_constraint_count(rb, W, no); }

template <class T> static T half_sq(const T* r, int m) {
  T s(0.0);
  for (int k = 0; k < m; ++k) s += r[k] * r[k];
  return T(0.5) * s;
}

// ---------------------------------------------------------------------------------------------
// Complex-step Jacobian of a residual function r(x): J[k][c] = Im r_k(x + i h e_c) / h.
// ---------------------------------------------------------------------------------------------
static const double CS_H = 1e-30;

typedef std::function<void(const cd* x, cd* r)> CResFn;

static void cs_jacobian(const CResFn& f, int nx, int nr, const double* x, double* J) {
  std::vector<cd> xc(nx), rc(nr);
  for (int c = 0; c < nx; ++c) {
    for (int q = 0; q < nx; ++q) xc[q] = cd(x[q], q == c ? CS_H : 0.0);
    f(xc.data(), rc.data());
    for (int k = 0; k < nr; ++k) J[k * nx + c] = rc[k].imag() / CS_H;
  }
}

// ---------------------------------------------------------------------------------------------
// Levenberg-Marquardt (Sec. IV-C): one iteration on a generic residual function.
// ---------------------------------------------------------------------------------------------

// Textbook Cholesky A = L L^T of a dense symmetric n x n matrix (row-major, lower part used).
// Returns false on a non-positive pivot. (Templated so that the op-counting scalar can count it.)
template <class T> static bool cholesky_t(int n, const T* A, T* Lm) {
  for (int i = 0; i < n * n; ++i) Lm[i] = T(0.0);
  for (int j = 0; j < n; ++j) {
    T s = A[j * n + j];
    for (int k = 0; k < j; ++k) s -= Lm[j * n + k] * Lm[j * n + k];
    if (!(re(s) > 0.0)) return false;
    T ljj = Sqrt(s);
    Lm[j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      T t = A[i * n + j];
      for (int k = 0; k < j; ++k) t -= Lm[i * n + k] * Lm[j * n + k];
      Lm[i * n + j] = t / ljj;
    }
  }
  return true;
}
static bool cholesky(int n, const double* A, double* Lm) { return cholesky_t<double>(n, A, Lm); }

// Solve L L^T x = b.
template <class T> static void chol_solve_t(int n, const T* Lm, const T* b, T* x) {
  std::vector<T> y(n);
  for (int i = 0; i < n; ++i) {
    T s = b[i];
    for (int k = 0; k < i; ++k) s -= Lm[i * n + k] * y[k];
    y[i] = s / Lm[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    T s = y[i];
    for (int k = i + 1; k < n; ++k) s -= Lm[k * n + i] * x[k];
    x[i] = s / Lm[i * n + i];
  }
}
static void chol_solve(int n, const double* Lm, const double* b, double* x) { chol_solve_t<double>(n, Lm, b, x); }

struct LmState {
  double lambda, nu, F;
  double Ftrial;  // cost at the trial point of the last iteration (NaN if its Cholesky failed)
  double Fstart;  // cost at the iterate the last iteration started from
};

// Steps 2-5 of one LM iteration, given F = F(x), A = J^T J (nx*nx, row-major, overwritten) and
// g = J^T r at x, and the cost function for the trial point:
//  2. A <- A + lambda D, D = diag(max(diag(J^T J), 1e-12)) (Marquardt scaling).
//  3. Cholesky of A; on a non-positive pivot: lambda <- lambda nu, nu <- 2 nu, x unchanged.
//  4. delta = -A^{-1} g; gain ratio rho = (F - F(x + delta)) / (1/2 delta^T (lambda D delta - g)).
//  5. Accept iff F(x + delta) < F: lambda <- lambda max(1/3, 1 - (2 rho - 1)^3), nu <- 2;
//     otherwise lambda <- lambda nu, nu <- 2 nu (Madsen, Nielsen and Tingleff 2004, Sec. 3.2).
// Every LM of the oracle (IK, calibration, the path's joint solve) goes through this one routine.
// Returns 1 if the step was accepted.
static int lm_update(int nx, double* A, const double* g, double F, const std::function<double(const double*)>& cost,
                     double* x, LmState& st) {
  std::vector<double> D(nx), Lm((size_t)nx * nx), delta(nx), xn(nx), mg(nx);
  st.F = F;
  st.Fstart = F;
  for (int a = 0; a < nx; ++a) {
    D[a] = std::max(A[(size_t)a * nx + a], 1e-12);
    A[(size_t)a * nx + a] += st.lambda * D[a];
  }
  if (!cholesky(nx, A, Lm.data())) {
    st.lambda *= st.nu;
    st.nu *= 2.0;
    st.Ftrial = NAN;
    return 0;
  }
  for (int a = 0; a < nx; ++a) mg[a] = -g[a];
  chol_solve(nx, Lm.data(), mg.data(), delta.data());
  for (int a = 0; a < nx; ++a) xn[a] = x[a] + delta[a];
  double Fn = cost(xn.data());
  st.Ftrial = Fn;
  double pred = 0;
  for (int a = 0; a < nx; ++a) pred += delta[a] * (st.lambda * D[a] * delta[a] - g[a]);
  pred *= 0.5;
  if (Fn < F) {
    double rho = (F - Fn) / pred;
    double t = 2.0 * rho - 1.0;
    st.lambda *= std::max(1.0 / 3.0, 1.0 - t * t * t);
    st.nu = 2.0;
    for (int a = 0; a < nx; ++a) x[a] = xn[a];
    st.F = Fn;
    return 1;
  }
  st.lambda *= st.nu;
  st.nu *= 2.0;
  return 0;
}

// One LM iteration (fixed-count schedule, no early exit) on a residual function:
//  1. r, J at x (complex-step J); F = 1/2 |r|^2; A = J^T J, g = J^T r.
//  2.-5. lm_update.
static int lm_iteration(const std::function<void(const double*, double*)>& fr, const CResFn& fc,
                        int nx, int nr, double* x, LmState& st) {
  std::vector<double> r(nr), J((size_t)nr * nx), A((size_t)nx * nx), g(nx), rn(nr);
  fr(x, r.data());
  double F = 0;
  for (int k = 0; k < nr; ++k) F += r[k] * r[k];
  F *= 0.5;
  cs_jacobian(fc, nx, nr, x, J.data());
  for (int a = 0; a < nx; ++a) {
    double s = 0;
    for (int k = 0; k < nr; ++k) s += J[(size_t)k * nx + a] * r[k];
    g[a] = s;
    for (int b = 0; b < nx; ++b) {
      double t = 0;
      for (int k = 0; k < nr; ++k) t += J[(size_t)k * nx + a] * J[(size_t)k * nx + b];
      A[a * nx + b] = t;
    }
  }
  auto cost = [&](const double* xx) {
    fr(xx, rn.data());
    double Fn = 0;
    for (int k = 0; k < nr; ++k) Fn += rn[k] * rn[k];
    return 0.5 * Fn;
  };
  return lm_update(nx, A.data(), g.data(), F, cost, x, st);
}

// ---------------------------------------------------------------------------------------------
// Projection onto the feasible tendon set of one segment (stage one of Algorithm 1)
// ---------------------------------------------------------------------------------------------

// Euclidean projection of v (m values) onto {|u_j| <= b, sum_j u_j = 0}. By the KKT conditions the
// projection is u_j = clamp(v_j - tau, -b, b) with tau the root of the non-increasing piecewise
// linear function g(tau) = sum_j clamp(v_j - tau, -b, b). The oracle sorts the 2m breakpoints
// v_j -/+ b, walks them until g changes sign and interpolates linearly on that piece.
static void project_segment(const double* v, int m, double b, double* u) {
  std::vector<double> bp;
  for (int j = 0; j < m; ++j) { bp.push_back(v[j] - b); bp.push_back(v[j] + b); }
  std::sort(bp.begin(), bp.end());
  auto g = [&](double tau) {
    double s = 0;
    for (int j = 0; j < m; ++j) s += std::min(b, std::max(-b, v[j] - tau));
    return s;
  };
  double tau = bp.back();
  for (size_t q = 0; q + 1 < bp.size(); ++q) {
    double g0 = g(bp[q]), g1 = g(bp[q + 1]);
    if (g0 >= 0.0 && g1 <= 0.0) {
      tau = (g0 == g1) ? bp[q] : bp[q] + g0 * (bp[q + 1] - bp[q]) / (g0 - g1);
      break;
    }
  }
  for (int j = 0; j < m; ++j) u[j] = std::min(b, std::max(-b, v[j] - tau));
}

// OR_MODEL_ARC: Euclidean projection onto {theta <= thmax} x [lmin, lmax] (a disk times an
// interval, so each factor projects on its own): the bend (tx, ty) is scaled back radially onto
// the disk, L is clamped.
static void project_arc(const double* v, double thmax, double lmin, double lmax, double* u) {
  const double r = std::sqrt(v[0] * v[0] + v[1] * v[1]);
  const double f = r > thmax ? thmax / r : 1.0;
  u[0] = v[0] * f;
  u[1] = v[1] * f;
  u[2] = std::min(lmax, std::max(lmin, v[2]));
}

static void project_state(const OrRobot& rb, const double* v, double* u) {
  for (int i = 0; i < rb.n; ++i) {
    if (rb.model == OR_MODEL_ARC) project_arc(v + 3 * i, rb.thmax[i], rb.lmin[i], rb.lmax[i], u + 3 * i);
    else project_segment(v + rb.m * i, rb.m, rb.umax[i], u + rb.m * i);
  }
}

// ---------------------------------------------------------------------------------------------
// Seeds (SampleSeeds of Algorithm 1): counter-based SplitMix64 and hexagon-uniform draws.
// ---------------------------------------------------------------------------------------------

// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): the k-th output from state s0 is
// mix(s0 + k * 0x9E3779B97F4A7C15), mix = the variant-13 finaliser of MurmurHash3.
static uint64_t splitmix64_at(uint64_t s0, uint64_t k) {
  uint64_t z = s0 + k * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static double u01_from(uint64_t z) { return (double)(z >> 11) * (1.0 / 9007199254740992.0); }

// Counter of draw w (0..2) for problem p, seed s, attempt a (0..7), segment i (0..7).
static uint64_t seed_counter(uint64_t p, uint64_t s, uint64_t a, uint64_t i, uint64_t w) {
  return ((((p * 65536ULL + s) * 8ULL + a) * 8ULL + i) * 4ULL + w) + 1ULL;
}

// Uniform point of the hexagon {|u_j| <= b, sum u = 0} (m = 3): the hexagon with vertices
// V_0..V_5 = (b,0,-b), (b,-b,0), (0,-b,b), (-b,0,b), (-b,b,0), (0,b,-b) in cyclic order is the
// union of the three congruent rhombi {x V_2k + y V_2k+2 : x, y in [0,1]}, k = 0,1,2.
static void hexagon_point(double b, double U0, double U1, double U2, double* u) {
  static const int V[6][3] = {{1, 0, -1}, {1, -1, 0}, {0, -1, 1}, {-1, 0, 1}, {-1, 1, 0}, {0, 1, -1}};
  int k = (int)(3.0 * U0);
  if (k > 2) k = 2;
  const int* A = V[2 * k];
  const int* B = V[(2 * k + 2) % 6];
  for (int j = 0; j < 3; ++j) {
    double ta = A[j] == 0 ? 0.0 : (A[j] > 0 ? U1 * b : -(U1 * b));
    double tb = B[j] == 0 ? 0.0 : (B[j] > 0 ? U2 * b : -(U2 * b));
    u[j] = ta + tb;
  }
}

// OR_MODEL_ARC seed of one segment: L uniform on [lmin, lmax] (draw 0) and the bend (tx, ty)
// uniform on the disk of radius thmax by rejection from the enclosing square: try t = 0..7 draws
// the square's point from counters (draw 1 and draw 2) + t * 2^48 (beyond every draw counter of
// problems p < 2^24) and keeps the first inside; if none is, the last is scaled onto the circle.
static void arc_seed_point(uint64_t key, uint64_t p, uint64_t s, uint64_t a, uint64_t i, double thmax,
                           double lmin, double lmax, double* q) {
  const double UL = u01_from(splitmix64_at(key, seed_counter(p, s, a, i, 0)));
  double x = 0, y = 0;
  bool in = false;
  for (uint64_t t = 0; t < 8 && !in; ++t) {
    const double X = u01_from(splitmix64_at(key, seed_counter(p, s, a, i, 1) + (t << 48)));
    const double Y = u01_from(splitmix64_at(key, seed_counter(p, s, a, i, 2) + (t << 48)));
    x = (2.0 * X - 1.0) * thmax;
    y = (2.0 * Y - 1.0) * thmax;
    in = x * x + y * y <= thmax * thmax;
  }
  if (!in) {
    const double f = thmax / std::sqrt(x * x + y * y);
    x = x * f;
    y = y * f;
  }
  q[0] = x;
  q[1] = y;
  q[2] = lmin + UL * (lmax - lmin);
}

// ---------------------------------------------------------------------------------------------
// Batch helpers
// ---------------------------------------------------------------------------------------------

static void parallel_for(int64_t n, int threads, const std::function<void(int64_t)>& body) {
  if (threads <= 1 || n <= 1) {
    for (int64_t i = 0; i < n; ++i) body(i);
    return;
  }
  std::vector<std::thread> pool;
  int64_t chunk = (n + threads - 1) / threads;
  for (int t = 0; t < threads; ++t) {
    int64_t lo = t * chunk, hi = std::min(n, lo + chunk);
    if (lo >= hi) break;
    pool.emplace_back([lo, hi, &body]() {
      for (int64_t i = lo; i < hi; ++i) body(i);
    });
  }
  for (auto& th : pool) th.join();
}

// IK residual closures for one seed.
struct IkProblem {
  const OrRobot* rb;
  const OrWeights* W;
  int no;
  const double* obs;
  int kind;
  const double* tgt;
  int d() const { return rb->n * rb->m; }
  int rows() const { return ik_rows(*rb, *W, no); }
  void res(const double* u, double* r) const {
    Params<double> P = params_of<double>(*rb);
    ik_residual(*rb, P, *W, no, obs, kind, tgt, u, r, (double*)nullptr);
  }
  void cres(const cd* u, cd* r) const {
    Params<cd> P = params_of<cd>(*rb);
    ik_residual(*rb, P, *W, no, obs, kind, tgt, u, r, (cd*)nullptr);
  }
  double cost(const double* u, double* coll) const {
    std::vector<double> r(rows());
    Params<double> P = params_of<double>(*rb);
    double cp = 0;
    ik_residual(*rb, P, *W, no, obs, kind, tgt, u, r.data(), &cp);
    if (coll) *coll = 0.5 * cp;
    return half_sq(r.data(), rows());
  }
  // gradient of the cost = J^T r
  void grad(const double* u, double* g) const {
    int nr = rows(), nx = d();
    std::vector<double> r(nr), J((size_t)nr * nx);
    res(u, r.data());
    cs_jacobian([this](const cd* x, cd* rr) { cres(x, rr); }, nx, nr, u, J.data());
    for (int a = 0; a < nx; ++a) {
      double s = 0;
      for (int k = 0; k < nr; ++k) s += J[(size_t)k * nx + a] * r[k];
      g[a] = s;
    }
  }
};

// Stage-one projected-gradient rule (normalised gradient step with an adaptive length alpha), on
// any cost F with gradient grad and feasible-set projection Pi:
//   trial x' = Pi(x - alpha g / |g|) (no move when g = 0);
//   accept iff F(x') < F(x): then x <- x', g <- grad F(x'), alpha <- 1.25 alpha;
//   otherwise x (and its g) stay and alpha <- alpha / 2.
// A fixed number of steps. Stage one of Algorithm 1 (per seed) and the trajectory refinement (all
// free states at once, the norm over all of them) both run this one routine. hist (nullable)
// receives, after every step, x, then alpha, F and the trial's cost F(x'): [steps][nx + 3].
// The step of the rule before the projection: v = x - alpha g / |g| (v = x when g = 0). A template so
// that the op-counting scalar counts this very code.
template <class T> static void pg_direction(int nx, const T* x, const T* g, T alpha, T* v) {
  T gn = T(0);
  for (int a = 0; a < nx; ++a) gn += g[a] * g[a];
  gn = Sqrt(gn);
  const T scale = re(gn) > 0 ? alpha / gn : T(0);
  for (int a = 0; a < nx; ++a) v[a] = x[a] - scale * g[a];
}

static void pg_rule(int nx, double* x, int steps, double alpha0, const std::function<double(const double*)>& cost,
                    const std::function<void(const double*, double*)>& grad,
                    const std::function<void(const double*, double*)>& project, double* F_out, double* hist) {
  std::vector<double> g(nx), x1(nx), v(nx), g1(nx);
  double F = cost(x);
  grad(x, g.data());
  double alpha = alpha0;
  for (int it = 0; it < steps; ++it) {
    pg_direction<double>(nx, x, g.data(), alpha, v.data());
    project(v.data(), x1.data());
    const double F1 = cost(x1.data());
    if (F1 < F) {
      grad(x1.data(), g1.data());
      for (int a = 0; a < nx; ++a) { x[a] = x1[a]; g[a] = g1[a]; }
      F = F1;
      alpha *= 1.25;
    } else {
      alpha *= 0.5;
    }
    if (hist) {
      double* h = hist + (size_t)it * (nx + 3);
      for (int a = 0; a < nx; ++a) h[a] = x[a];
      h[nx] = alpha;
      h[nx + 1] = F;
      h[nx + 2] = F1;
    }
  }
  if (F_out) *F_out = F;
}

// Stage one of Algorithm 1 for one seed: pg_rule on its IK cost, projected per segment.
static void pg_run_one(const IkProblem& pb, double* u, int steps, double alpha0, double* F_out,
                       double* hist = nullptr) {
  const OrRobot& rb = *pb.rb;
  pg_rule(pb.d(), u, steps, alpha0, [&pb](const double* x) { return pb.cost(x, nullptr); },
          [&pb](const double* x, double* g) { pb.grad(x, g); },
          [&rb](const double* v, double* x1) { project_state(rb, v, x1); }, F_out, hist);
}

// ---------------------------------------------------------------------------------------------
// Exported C API (row-major AoS arrays; B = batch of states)
// ---------------------------------------------------------------------------------------------
extern "C" {

int orc_version() { return 1; }

// Forward kinematics: T_out[B][12] = R row-major (9) then p (3); backbone[B][n*nb][3] or null.
int orc_fk(const OrRobot* rb, const double* u, int64_t B, double* T_out, double* backbone) {
  int d = rb->n * rb->m;
  Params<double> P = params_of<double>(*rb);
  for (int64_t b = 0; b < B; ++b) {
    FkOut<double> o;
    forward_kinematics(*rb, P, u + d * b, o, backbone ? backbone + (size_t)3 * rb->n * rb->nb * b : nullptr);
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 3; ++c) T_out[12 * b + 3 * a + c] = o.R[a][c];
    for (int a = 0; a < 3; ++a) T_out[12 * b + 9 + a] = o.p[a];
  }
  return 0;
}

// Same, with the minimal (Rodrigues) arithmetic form of Eq. 2-3 instead of the ZYZ product.
int orc_fk_rodrigues(const OrRobot* rb, const double* u, int64_t B, double* T_out) {
  g_count_minimal = true;
  int rc = orc_fk(rb, u, B, T_out, nullptr);
  g_count_minimal = false;
  return rc;
}

// Tendon map: (theta, phi) of every segment, and Eq. 4 forward for round trips.
int orc_bend(const OrRobot* rb, const double* u, int64_t B, double* theta_phi /*[B][n][2]*/) {
  int d = rb->n * rb->m;
  for (int64_t b = 0; b < B; ++b)
    for (int i = 0; i < rb->n; ++i) {
      double tx, ty;
      tendon_to_bend(u + d * b + rb->m * i, rb->m, rb->rc[i], tx, ty);
      theta_phi[2 * (rb->n * b + i)] = std::sqrt(tx * tx + ty * ty);
      theta_phi[2 * (rb->n * b + i) + 1] = std::atan2(ty, tx);
    }
  return 0;
}
int orc_tendon_lengths(double rc, double L, double theta, double phi, int m, double* l_out) {
  for (int j = 0; j < m; ++j) l_out[j] = L + tendon_displacement(rc, theta, phi, j, m);
  return 0;
}

// Tip Jacobian [B][6][d]: rows 0-2 d p / d u, rows 3-5 the world angular velocity
// vee(dR R^T) per unit du, by complex step on the forward kinematics.
int orc_tip_jacobian(const OrRobot* rb, const double* u, int64_t B, double* J) {
  int d = rb->n * rb->m;
  Params<cd> P = params_of<cd>(*rb);
  Params<double> Pd = params_of<double>(*rb);
  for (int64_t b = 0; b < B; ++b) {
    FkOut<double> o;
    forward_kinematics(*rb, Pd, u + d * b, o, nullptr);
    for (int c = 0; c < d; ++c) {
      std::vector<cd> x(d);
      for (int q = 0; q < d; ++q) x[q] = cd(u[d * b + q], q == c ? CS_H : 0.0);
      FkOut<cd> oc;
      forward_kinematics(*rb, P, x.data(), oc, nullptr);
      double dR[3][3];
      for (int a = 0; a < 3; ++a) {
        J[(size_t)6 * d * b + a * d + c] = oc.p[a].imag() / CS_H;
        for (int e = 0; e < 3; ++e) dR[a][e] = oc.R[a][e].imag() / CS_H;
      }
      double Wm[3][3];  // dR R^T
      for (int a = 0; a < 3; ++a)
        for (int e = 0; e < 3; ++e) {
          double s = 0;
          for (int k = 0; k < 3; ++k) s += dR[a][k] * o.R[e][k];
          Wm[a][e] = s;
        }
      J[(size_t)6 * d * b + 3 * d + c] = 0.5 * (Wm[2][1] - Wm[1][2]);
      J[(size_t)6 * d * b + 4 * d + c] = 0.5 * (Wm[0][2] - Wm[2][0]);
      J[(size_t)6 * d * b + 5 * d + c] = 0.5 * (Wm[1][0] - Wm[0][1]);
    }
  }
  return 0;
}

int orc_so3_log(const double* E /*[B][9]*/, int64_t B, double* w /*[B][3]*/) {
  for (int64_t b = 0; b < B; ++b) {
    double M[3][3];
    for (int a = 0; a < 9; ++a) M[a / 3][a % 3] = E[9 * b + a];
    so3_log(M, w + 3 * b);
  }
  return 0;
}

// Signed distance sd of points x [B][3] to the core of obstacle record ob [OR_OBS], and with
// grad != NULL its gradient d sd / dx [B][3] (complex step).
int orc_obstacle_sd(const double* ob, const double* x, int64_t B, double* sd, double* grad) {
  for (int64_t b = 0; b < B; ++b) {
    sd[b] = obstacle_sd(ob, x + 3 * b);
    if (!grad) continue;
    for (int a = 0; a < 3; ++a) {
      cd xc[3] = {x[3 * b], x[3 * b + 1], x[3 * b + 2]};
      xc[a] += cd(0.0, 1e-30);
      grad[3 * b + a] = obstacle_sd(ob, xc).imag() / 1e-30;
    }
  }
  return 0;
}

int orc_quat_to_R(const double* q, int64_t B, double* R /*[B][9]*/) {
  for (int64_t b = 0; b < B; ++b) {
    double M[3][3];
    quat_to_R(q + 4 * b, M);
    for (int a = 0; a < 9; ++a) R[9 * b + a] = M[a / 3][a % 3];
  }
  return 0;
}

int orc_ik_rows(const OrRobot* rb, const OrWeights* W, int no) { return ik_rows(*rb, *W, no); }

// IK residuals r[B][rows], cost F[B], collision part of the cost coll[B] (nullable), gradient
// g[B][d] (nullable) and residual Jacobian J[B][rows][d] (nullable). Target of seed b is
// targets[7 * (b / S)].
int orc_ik_eval(const OrRobot* rb, const OrWeights* W, int no, const double* obs, int kind,
                const double* targets, int64_t S, const double* u, int64_t B, double* r, double* F,
                double* coll, double* g, double* J, int threads) {
  int d = rb->n * rb->m;
  parallel_for(B, threads, [&](int64_t b) {
    IkProblem pb{rb, W, no, obs, kind, targets + 7 * (b / S)};
    int nr = pb.rows();
    std::vector<double> rr(nr);
    pb.res(u + d * b, rr.data());
    if (r) std::memcpy(r + (size_t)nr * b, rr.data(), sizeof(double) * nr);
    if (F) F[b] = pb.cost(u + d * b, coll ? coll + b : nullptr);
    else if (coll) pb.cost(u + d * b, coll + b);
    if (g) pb.grad(u + d * b, g + (size_t)d * b);
    if (J)
      cs_jacobian([&pb](const cd* x, cd* rc) { pb.cres(x, rc); }, d, nr, u + d * b,
                  J + (size_t)nr * d * b);
  });
  return 0;
}

// Gradient of the summed IK cost with respect to the kinematic parameters (L_i, r_c,i),
// complex step on each parameter: grad[2n] = d/dL_1..n then d/dr_c,1..n of sum_b F_b.
int orc_ik_param_grad(const OrRobot* rb, const OrWeights* W, int no, const double* obs,
                      int kind, const double* targets, int64_t S, const double* u, int64_t B,
                      double* grad) {
  int d = rb->n * rb->m;
  for (int q = 0; q < 2 * rb->n; ++q) {
    double acc = 0;
    for (int64_t b = 0; b < B; ++b) {
      Params<cd> P = params_of<cd>(*rb);
      if (q < rb->n) P.L[q] += cd(0.0, CS_H);
      else P.rc[q - rb->n] += cd(0.0, CS_H);
      int nr = ik_rows(*rb, *W, no);
      std::vector<cd> x(d), r(nr);
      for (int a = 0; a < d; ++a) x[a] = cd(u[d * b + a], 0.0);
      ik_residual(*rb, P, *W, no, obs, kind, targets + 7 * (b / S), x.data(), r.data(), (cd*)nullptr);
      cd F = half_sq(r.data(), nr);
      acc += F.imag() / CS_H;
    }
    grad[q] = acc;
  }
  return 0;
}

// Run `iters` LM iterations on each seed. u[B][d] is updated in place; hist (nullable) receives
// the iterate after every iteration [iters][B][d]; lam/nu/F (in/out, [B]); acc[B][iters] (nullable)
// the accept flags; trace[B][iters][2] (nullable) the cost at the iteration's start and at its trial
// point. lam/nu must be initialised by the caller (lambda0, 2).
int orc_ik_lm(const OrRobot* rb, const OrWeights* W, int no, const double* obs, int kind,
              const double* targets, int64_t S, double* u, int64_t B, int iters, double* lam,
              double* nu, double* F, double* hist, uint8_t* acc, double* trace, int threads) {
  int d = rb->n * rb->m;
  parallel_for(B, threads, [&](int64_t b) {
    IkProblem pb{rb, W, no, obs, kind, targets + 7 * (b / S)};
    LmState st{lam[b], nu[b], 0.0, 0.0, 0.0};
    double* x = u + d * b;
    for (int it = 0; it < iters; ++it) {
      int a = lm_iteration([&pb](const double* xx, double* rr) { pb.res(xx, rr); },
                           [&pb](const cd* xx, cd* rr) { pb.cres(xx, rr); }, d, pb.rows(), x, st);
      if (acc) acc[(size_t)iters * b + it] = (uint8_t)a;
      if (hist) std::memcpy(hist + ((size_t)it * B + b) * d, x, sizeof(double) * d);
      if (trace) {
        trace[((size_t)iters * b + it) * 2] = st.Fstart;
        trace[((size_t)iters * b + it) * 2 + 1] = st.Ftrial;
      }
    }
    lam[b] = st.lambda;
    nu[b] = st.nu;
    F[b] = pb.cost(x, nullptr);
  });
  return 0;
}

// LM on a linear residual r(x) = A x - y (A is [nr][nx]); used to pin the LM machinery.
int orc_lm_linear(const double* A, const double* y, int nr, int nx, double* x, int iters,
                  double* lam, double* nu, double* F) {
  auto fr = [&](const double* xx, double* rr) {
    for (int k = 0; k < nr; ++k) {
      double s = -y[k];
      for (int a = 0; a < nx; ++a) s += A[k * nx + a] * xx[a];
      rr[k] = s;
    }
  };
  auto fc = [&](const cd* xx, cd* rr) {
    for (int k = 0; k < nr; ++k) {
      cd s = -y[k];
      for (int a = 0; a < nx; ++a) s += A[k * nx + a] * xx[a];
      rr[k] = s;
    }
  };
  LmState st{*lam, *nu, 0.0};
  for (int it = 0; it < iters; ++it) lm_iteration(fr, fc, nx, nr, x, st);
  *lam = st.lambda;
  *nu = st.nu;
  std::vector<double> r(nr);
  fr(x, r.data());
  double s = 0;
  for (int k = 0; k < nr; ++k) s += r[k] * r[k];
  *F = 0.5 * s;
  return 0;
}

// Pins of the step rules on problems that can be solved by hand.
// pg_rule on F(u) = 1/2 |u - c|^2 (gradient u - c) over nseg hexagons {|u_j| <= b_i, sum_j u_j = 0}
// (three tendons per segment); hist as in pg_rule, [steps][3 nseg + 3].
int orc_pg_quadratic(const double* c, int nseg, const double* b, double* u, int steps, double alpha0, double* F,
                     double* hist) {
  const int nx = 3 * nseg;
  pg_rule(nx, u, steps, alpha0,
          [c, nx](const double* x) {
            double s = 0;
            for (int a = 0; a < nx; ++a) s += (x[a] - c[a]) * (x[a] - c[a]);
            return 0.5 * s;
          },
          [c, nx](const double* x, double* g) {
            for (int a = 0; a < nx; ++a) g[a] = x[a] - c[a];
          },
          [b, nseg](const double* v, double* x1) {
            for (int i = 0; i < nseg; ++i) project_segment(v + 3 * i, 3, b[i], x1 + 3 * i);
          },
          F, hist);
  return 0;
}

// lm_iteration on the scalar residual r(x) = x^2 - a; after every iteration: x, lambda, nu, F (the
// cost at the iterate the iteration started from) and the accept flag.
int orc_lm_scalar(double a, double x0, int iters, double lambda0, double* x_hist, double* lam_hist,
                  double* nu_hist, double* F_hist, uint8_t* acc) {
  auto fr = [a](const double* xx, double* rr) { rr[0] = xx[0] * xx[0] - a; };
  auto fc = [a](const cd* xx, cd* rr) { rr[0] = xx[0] * xx[0] - a; };
  LmState st{lambda0, 2.0, 0.0};
  double x = x0;
  for (int it = 0; it < iters; ++it) {
    double Fstart = 0.5 * (x * x - a) * (x * x - a);
    acc[it] = (uint8_t)lm_iteration(fr, fc, 1, 1, &x, st);
    x_hist[it] = x;
    lam_hist[it] = st.lambda;
    nu_hist[it] = st.nu;
    F_hist[it] = Fstart;
  }
  return 0;
}

// The op-counting scalar on small programs whose counts are known by hand (out as orc_opcount_ik):
//   which 0: C = A B of two 3x3 matrices that both depend on the input;
//   which 1: C = A B with only A depending on it;
//   which 2: y = sum_{k<5} a_k x_k, a linear function with constant a_k;
//   which 3: one segment of Eq. 2-3 in the minimal (Rodrigues) form, (tx, ty) the input, L constant;
//   which 4: y = sin(x) cos(x) / sqrt(x).
// Op count of the step of one projected-gradient iteration (pg_direction: the gradient norm, the
// step length and the move) on nx unknowns, without the projection (comparisons and clamps) and the
// cost evaluation (forward flops and special calls in out[0..1]).
int orc_opcount_pg_step(int nx, long long* out) {
  g_tally = {0, 0, 0, 0};
  std::vector<Cnt> x(nx), g(nx), v(nx);
  for (int a = 0; a < nx; ++a) { x[a] = Cnt(1e-3 * (a + 1)); g[a] = Cnt(0.5 - 0.1 * a); }
  pg_direction<Cnt>(nx, x.data(), g.data(), Cnt(1e-3), v.data());
  out[0] = g_tally.f_flop;
  out[1] = g_tally.f_sfu;
  return 0;
}

// Op count of steps 2-5 of one LM iteration (lm_update) on nx unknowns, without the cost
// evaluations: damping of the diagonal, Cholesky, the two triangular solves, the predicted
// decrease, the gain ratio and the damping update (forward flops and special calls in out[0..1]).
int orc_opcount_lm_update(int nx, long long* out) {
  g_tally = {0, 0, 0, 0};
  std::vector<Cnt> A((size_t)nx * nx), Lm((size_t)nx * nx), g(nx), D(nx), mg(nx), dl(nx);
  for (int a = 0; a < nx; ++a)
    for (int b = 0; b < nx; ++b) A[(size_t)a * nx + b] = Cnt(a == b ? 2.0 + a : 0.1 / (1 + a + b));
  for (int a = 0; a < nx; ++a) g[a] = Cnt(0.5 - 0.1 * a);
  const Cnt lam(1e-3);
  for (int a = 0; a < nx; ++a) {
    D[a] = A[(size_t)a * nx + a];  // max(diag, 1e-12): a comparison, not counted
    A[(size_t)a * nx + a] += lam * D[a];
  }
  cholesky_t<Cnt>(nx, A.data(), Lm.data());
  for (int a = 0; a < nx; ++a) mg[a] = -g[a];
  chol_solve_t<Cnt>(nx, Lm.data(), mg.data(), dl.data());
  Cnt pred(0.0);
  for (int a = 0; a < nx; ++a) pred += dl[a] * (lam * D[a] * dl[a] - g[a]);
  pred *= Cnt(0.5);
  const Cnt F(1.0), Fn(0.5);
  const Cnt rho = (F - Fn) / pred;
  const Cnt t = Cnt(2.0) * rho - Cnt(1.0);
  Cnt lam2 = lam * (Cnt(1.0) - t * t * t);
  (void)lam2;
  out[0] = g_tally.f_flop;
  out[1] = g_tally.f_sfu;
  return 0;
}

int orc_opcount_probe(int which, long long* out) {
  g_tally = {0, 0, 0, 0};
  if (which == 0 || which == 1) {
    Cnt A[3][3], B[3][3], Cm[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        A[i][j] = Cnt(1.0 + i + 0.5 * j, true);
        B[i][j] = Cnt(2.0 - j + 0.25 * i, which == 0);
      }
    matmul3(A, B, Cm);
  } else if (which == 2) {
    Cnt y(0.0);
    Cnt x[5];
    for (int k = 0; k < 5; ++k) x[k] = Cnt(0.1 * (k + 1), true);
    y = Cnt(0.5) * x[0];
    for (int k = 1; k < 5; ++k) y = y + Cnt(0.5 + k) * x[k];
  } else if (which == 3) {
    g_count_minimal = true;
    Cnt R[3][3], d[3];
    segment_transform(Cnt(0.3, true), Cnt(-0.2, true), Cnt(0.1), R, d);
    g_count_minimal = false;
  } else if (which == 4) {
    Cnt x(0.7, true);
    Cnt y = Sin(x) * Cos(x) / Sqrt(x);
    (void)y;
  } else {
    return 1;
  }
  out[0] = g_tally.f_flop;
  out[1] = g_tally.f_sfu;
  out[2] = g_tally.t_flop;
  out[3] = g_tally.t_sfu;
  return 0;
}

int orc_cholesky(int n, const double* A, double* Lm) { return cholesky(n, A, Lm) ? 0 : 1; }

int orc_project(const double* v, int64_t B, int m, double b, double* u) {
  for (int64_t q = 0; q < B; ++q) project_segment(v + m * q, m, b, u + m * q);
  return 0;
}

// OR_MODEL_ARC projection of B segment states v[B][3] onto {theta <= thmax} x [lmin, lmax].
int orc_project_arc(const double* v, int64_t B, double thmax, double lmin, double lmax, double* u) {
  for (int64_t q = 0; q < B; ++q) project_arc(v + 3 * q, thmax, lmin, lmax, u + 3 * q);
  return 0;
}

// Stage-one projected gradient on every seed: u[B][d] in place, F[B] out; hist (nullable)
// [B][steps][d + 3] as in pg_rule.
// alpha_per (nullable): seed b starts with step length alpha_per[b] instead of alpha0.
int orc_ik_pg(const OrRobot* rb, const OrWeights* W, int no, const double* obs, int kind,
              const double* targets, int64_t S, double* u, int64_t B, int steps, double alpha0,
              const double* alpha_per, double* F, double* hist, int threads) {
  int d = rb->n * rb->m;
  parallel_for(B, threads, [&](int64_t b) {
    IkProblem pb{rb, W, no, obs, kind, targets + 7 * (b / S)};
    pg_run_one(pb, u + d * b, steps, alpha_per ? alpha_per[b] : alpha0, F + b,
               hist ? hist + (size_t)b * steps * (d + 3) : nullptr);
  });
  return 0;
}

uint64_t orc_splitmix64_at(uint64_t s0, uint64_t k) { return splitmix64_at(s0, k); }

// Seeds of problem p (global index p0 + q): u[P][S][d]. With obstacles, a seed with a backbone sample
// closer than r_o + r_body + delta to an obstacle's core is redrawn (attempts 0..7; the last draw is
// kept).
int orc_seeds(const OrRobot* rb, const OrWeights* W, int no, const double* obs, uint64_t base,
              int64_t p0, int64_t P, int64_t S, double* u) {
  int d = rb->n * rb->m;
  Params<double> Pd = params_of<double>(*rb);
  for (int64_t q = 0; q < P; ++q)
    for (int64_t s = 0; s < S; ++s) {
      double* x = u + ((size_t)q * S + s) * d;
      for (int a = 0; a < 8; ++a) {
        for (int i = 0; i < rb->n; ++i) {
          if (rb->model == OR_MODEL_ARC) {
            arc_seed_point(base, p0 + q, s, a, i, rb->thmax[i], rb->lmin[i], rb->lmax[i], x + 3 * i);
            continue;
          }
          double U[3];
          for (int w = 0; w < 3; ++w)
            U[w] = u01_from(splitmix64_at(base, seed_counter(p0 + q, s, a, i, w)));
          hexagon_point(rb->umax[i], U[0], U[1], U[2], x + 3 * i);
        }
        if (no == 0) break;
        FkOut<double> o;
        std::vector<double> bb(3 * rb->n * rb->nb);
        forward_kinematics(*rb, Pd, x, o, bb.data());
        bool hit = false;
        for (int k = 0; k < rb->n * rb->nb && !hit; ++k)
          for (int c = 0; c < no && !hit; ++c) {
            const double* ob = obs + OR_OBS * c;
            double sd;
            if (obstacle_within(ob, &bb[3 * k], ob[1] + rb->rbody + W->delta, sd)) hit = true;
          }
        if (!hit) break;
      }
    }
  return 0;
}

// SelectTop of Algorithm 1 for one problem: candidates ranked by (cost, collision penalty, index)
// ascending (non-finite costs last); a candidate within dedup_eps (max-norm) of an already kept
// one is skipped; if fewer than k survive, the best skipped candidates fill the rest in rank
// order. Keys are float32 so that both implementations decide in the same precision.
int orc_topk(const float* cost, const float* coll, const double* u /*[S][d]*/, int64_t S, int d,
             int k, double dedup_eps, int32_t* out) {
  std::vector<int> idx(S);
  for (int q = 0; q < S; ++q) idx[q] = q;
  auto key = [&](int q) { return std::isfinite(cost[q]) ? cost[q] : INFINITY; };
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
    float ka = key(a), kb = key(b);
    if (ka != kb) return ka < kb;
    if (coll[a] != coll[b]) return coll[a] < coll[b];
    return a < b;
  });
  std::vector<int> kept, skipped;
  for (int q : idx) {
    if ((int)kept.size() == k) break;
    bool dup = false;
    for (int c : kept) {
      double mx = 0;
      for (int a = 0; a < d; ++a) mx = std::max(mx, std::fabs(u[(size_t)q * d + a] - u[(size_t)c * d + a]));
      if (mx < dedup_eps) { dup = true; break; }
    }
    if (dup) skipped.push_back(q);
    else kept.push_back(q);
  }
  for (size_t q = 0; kept.size() < (size_t)k && q < skipped.size(); ++q) kept.push_back(skipped[q]);
  for (int q = 0; q < k; ++q) out[q] = q < (int)kept.size() ? kept[q] : -1;
  return 0;
}

// Final acceptance of one solution: position error (m), rotation error (rad: Log angle for IK6,
// angle between tip axes for IK5), limits (|u| <= umax + tol, |sum u| <= tol, or for OR_MODEL_ARC
// lmin - tol <= L <= lmax + tol; theta <= thmax + tol)
// and collision-free (every sample at least r_o + r_body from every obstacle's core).
// With self_check, collision-free also requires every pair of samples of segments two or more
// apart to be at least 2 r_body apart (the self-contact rows' reading, without the margin delta).
static void accept_one(const OrRobot& rb, int no, const double* obs, int kind,
                       const double* tgt, const double* u, double tol, double* pos, double* rot,
                       uint8_t* lim_ok, uint8_t* col_ok, bool self_check = false) {
  Params<double> Pd = params_of<double>(rb);
  FkOut<double> o;
  std::vector<double> bb(3 * rb.n * rb.nb);
  forward_kinematics(rb, Pd, u, o, bb.data());
  double dp2 = 0;
  for (int a = 0; a < 3; ++a) dp2 += (o.p[a] - tgt[a]) * (o.p[a] - tgt[a]);
  *pos = std::sqrt(dp2);
  if (kind == OR_IK5) {
    double zn = std::sqrt(tgt[3] * tgt[3] + tgt[4] * tgt[4] + tgt[5] * tgt[5]);
    double z[3] = {o.R[0][2], o.R[1][2], o.R[2][2]}, zt[3] = {tgt[3] / zn, tgt[4] / zn, tgt[5] / zn};
    double cx = z[1] * zt[2] - z[2] * zt[1], cy = z[2] * zt[0] - z[0] * zt[2], cz = z[0] * zt[1] - z[1] * zt[0];
    *rot = std::atan2(std::sqrt(cx * cx + cy * cy + cz * cz), z[0] * zt[0] + z[1] * zt[1] + z[2] * zt[2]);
  } else {
    double Rt[3][3], E[3][3], w[3];
    quat_to_R(tgt + 3, Rt);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) E[a][b] = Rt[0][a] * o.R[0][b] + Rt[1][a] * o.R[1][b] + Rt[2][a] * o.R[2][b];
    so3_log(E, w);
    *rot = std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
  }
  bool ok = true;
  for (int i = 0; i < rb.n; ++i) {
    if (rb.model == OR_MODEL_ARC) {
      const double L = u[3 * i + 2];
      if (L > rb.lmax[i] + tol || L < rb.lmin[i] - tol) ok = false;
    } else {
      double s = 0;
      for (int j = 0; j < rb.m; ++j) {
        double x = u[rb.m * i + j];
        s += x;
        if (std::fabs(x) > rb.umax[i] + tol) ok = false;
      }
      if (std::fabs(s) > tol) ok = false;
    }
    if (std::sqrt(o.th2[i]) > rb.thmax[i] + 1e-6) ok = false;
  }
  *lim_ok = ok;
  bool free = true;
  for (int k = 0; k < rb.n * rb.nb && free; ++k)
    for (int c = 0; c < no && free; ++c) {
      const double* ob = obs + OR_OBS * c;
      double sd;
      if (obstacle_within(ob, &bb[3 * k], ob[1] + rb.rbody, sd)) free = false;
    }
  if (self_check) {
    const double g2 = 4.0 * rb.rbody * rb.rbody;
    for (int i = 0; i < rb.n && free; ++i)
      for (int j = i + 2; j < rb.n && free; ++j)
        for (int ka = 0; ka < rb.nb && free; ++ka)
          for (int kb = 0; kb < rb.nb && free; ++kb) {
            const double* pa = &bb[3 * (i * rb.nb + ka)];
            const double* pb = &bb[3 * (j * rb.nb + kb)];
            const double dx = pa[0] - pb[0], dy = pa[1] - pb[1], dz = pa[2] - pb[2];
            if (dx * dx + dy * dy + dz * dz < g2) free = false;
          }
  }
  *col_ok = free;
}

// Cost below which refined candidates count as equally good solutions in the argmin of Algorithm 1
// (about 8 um of tip position under the default pose weights): their differences are rounding.
static const double OR_ARGMIN_TIE = 1e-8;

struct OrIkParams {
  int32_t S, n_final, k_init, k_final;
  double lambda0, alpha0, dedup_eps, lim_tol, pos_tol, rot_tol;
  uint64_t seed;
  int64_t p0;  // global index of the first problem (seed counter)
};

// Algorithm 1 per problem. Outputs u_out[P][d], F_out[P], pos[P], rot[P], success[P];
// cand_out (nullable) [P][n_final] the SelectTop indices; stage1_F (nullable) [P][S].
int orc_solve_ik(const OrRobot* rb, const OrWeights* W, int no, const double* obs, int kind,
                 const double* targets, int64_t P, const OrIkParams* prm, double* u_out,
                 double* F_out, double* pos, double* rot, uint8_t* success, int32_t* cand_out,
                 double* stage1_F, int threads) {
  int d = rb->n * rb->m;
  int S = prm->S, K = prm->n_final;
  parallel_for(P, threads, [&](int64_t q) {
    const double* tgt = targets + 7 * q;
    IkProblem pb{rb, W, no, obs, kind, tgt};
    std::vector<double> U((size_t)S * d), F(S), C(S);
    orc_seeds(rb, W, no, obs, prm->seed, prm->p0 + q, 1, S, U.data());
    // Stage one (ParallelOptimize with k_init steps): projected gradient on every seed.
    for (int s = 0; s < S; ++s) {
      if (prm->k_init > 0) pg_run_one(pb, U.data() + (size_t)s * d, prm->k_init, prm->alpha0, &F[s]);
      F[s] = pb.cost(U.data() + (size_t)s * d, &C[s]);
    }
    if (stage1_F)
      for (int s = 0; s < S; ++s) stage1_F[(size_t)q * S + s] = F[s];
    // SelectTop: keys in float32.
    std::vector<float> Ff(S), Cf(S);
    for (int s = 0; s < S; ++s) { Ff[s] = (float)F[s]; Cf[s] = (float)C[s]; }
    std::vector<int32_t> top(K);
    orc_topk(Ff.data(), Cf.data(), U.data(), S, d, K, prm->dedup_eps, top.data());
    if (cand_out)
      for (int c = 0; c < K; ++c) cand_out[(size_t)q * K + c] = top[c];
    // Stage two (ParallelOptimize with k_final LM iterations) and argmin of the final cost. Costs
    // at or below OR_ARGMIN_TIE are solutions whose differences are rounding: they count as equal
    // and the first of them in SelectTop order is kept; above it the lowest cost wins.
    double bestKey = INFINITY, bestF = INFINITY;
    int best = -1;
    std::vector<double> X((size_t)K * d);
    for (int c = 0; c < K; ++c) {
      double* x = X.data() + (size_t)c * d;
      if (top[c] < 0) { for (int a = 0; a < d; ++a) x[a] = NAN; continue; }
      std::memcpy(x, U.data() + (size_t)top[c] * d, sizeof(double) * d);
      LmState st{prm->lambda0, 2.0, 0.0};
      for (int it = 0; it < prm->k_final; ++it)
        lm_iteration([&pb](const double* xx, double* rr) { pb.res(xx, rr); },
                     [&pb](const cd* xx, cd* rr) { pb.cres(xx, rr); }, d, pb.rows(), x, st);
      double Fc = pb.cost(x, nullptr);
      const double key = Fc <= OR_ARGMIN_TIE ? 0.0 : Fc;
      if (key < bestKey) { bestKey = key; bestF = Fc; best = c; }
    }
    double* uo = u_out + (size_t)q * d;
    if (best < 0) {
      for (int a = 0; a < d; ++a) uo[a] = NAN;
      F_out[q] = NAN; pos[q] = NAN; rot[q] = NAN; success[q] = 0;
      return;
    }
    std::memcpy(uo, X.data() + (size_t)best * d, sizeof(double) * d);
    F_out[q] = bestF;
    uint8_t lim_ok, col_ok;
    accept_one(*rb, no, obs, kind, tgt, uo, prm->lim_tol, &pos[q], &rot[q], &lim_ok, &col_ok, W->rho_s > 0.0);
    success[q] = (pos[q] <= prm->pos_tol && rot[q] <= prm->rot_tol && lim_ok && col_ok) ? 1 : 0;
  });
  return 0;
}

int orc_accept(const OrRobot* rb, int no, const double* obs, int kind, const double* targets,
               const double* u, int64_t P, double tol, double* pos, double* rot, uint8_t* lim_ok,
               uint8_t* col_ok, int self_check) {
  int d = rb->n * rb->m;
  for (int64_t q = 0; q < P; ++q)
    accept_one(*rb, no, obs, kind, targets + 7 * q, u + (size_t)d * q, tol, pos + q, rot + q,
               lim_ok + q, col_ok + q, self_check != 0);
  return 0;
}

// Algorithmic op counts of one IK state evaluation in the minimal (Rodrigues) arithmetic form:
// out[0..3] = forward flops, forward special-function calls, tangent flops, tangent special calls
// (the tangent map of the cost w.r.t. u; a reverse sweep transposes it with the same count).
// box = 0 counts the cost without the rows that vanish on stage one's feasible set (tendon model:
// bound and sum-zero rows; arc model: length and curvature rows), so a projected trial point needs
// none of them.
int orc_opcount_ik_form(const OrRobot* rb, const OrWeights* W, int no, const double* obs, int kind,
                        const double* target, const double* u, int box, long long* out) {
  int d = rb->n * rb->m;
  g_count_minimal = true;
  g_count_skip_box = !box;
  g_tally = {0, 0, 0, 0};
  Params<Cnt> P;
  for (int i = 0; i < rb->n; ++i) { P.L[i] = Cnt(rb->L[i]); P.rc[i] = Cnt(rb->rc[i]); }
  std::vector<Cnt> x(d), r(ik_rows(*rb, *W, no));
  for (int a = 0; a < d; ++a) x[a] = Cnt(u[a], true);
  const int rows = ik_residual(*rb, P, *W, no, obs, kind, target, x.data(), r.data(), (Cnt*)nullptr);
  Cnt F = half_sq(r.data(), rows);
  (void)F;
  g_count_minimal = false;
  g_count_skip_box = false;
  out[0] = g_tally.f_flop;
  out[1] = g_tally.f_sfu;
  out[2] = g_tally.t_flop;
  out[3] = g_tally.t_sfu;
  return 0;
}

int orc_opcount_ik(const OrRobot* rb, const OrWeights* W, int no, const double* obs, int kind,
                   const double* target, const double* u, long long* out) {
  return orc_opcount_ik_form(rb, W, no, obs, kind, target, u, 1, out);
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Generic LM iteration on a normal-equation callback (used where J is assembled blockwise)
// ---------------------------------------------------------------------------------------------

// normal(x, A, g) returns F(x) and fills A = J^T J (nx*nx, row-major) and g = J^T r; cost(x) = F.
// Steps 2-5 are lm_update's.
static int lm_iteration_ag(const std::function<double(const double*, double*, double*)>& normal,
                           const std::function<double(const double*)>& cost, int nx, double* x,
                           LmState& st) {
  std::vector<double> A((size_t)nx * nx), g(nx);
  double F = normal(x, A.data(), g.data());
  return lm_update(nx, A.data(), g.data(), F, cost, x, st);
}

// ---------------------------------------------------------------------------------------------
// Trajectory planning
// ---------------------------------------------------------------------------------------------

// Residual of one trajectory of Tn >= 2 states; u_0 = u_start is fixed and x holds u_1..u_{Tn-1}.
// Rows, for t = 1..Tn-1 in order: path length sqrt(w_len)(p_t - p_{t-1}) (3, a sum-of-squares
// reading of the length objective), tendon speed hinges sqrt(rho_v) max(0, +-(u_t - u_{t-1})/dt -
// v_max) (2d), the state rows of u_t; for t >= 2 the acceleration hinges sqrt(rho_a) max(0,
// +-(u_t - 2 u_{t-1} + u_{t-2})/dt^2 - a_max) (2d). Last, the goal pose rows (6, full pose) of
// u_{Tn-1}. Tendon lengths are L_i + u_ij with fixed L_i, so tendon speeds are differences of u.
template <class T>
static int traj_residual(const OrRobot& rb, const Params<T>& P, const OrWeights& W, int no,
                         const double* obs, const double* u_start, const double* goal, int Tn,
                         const T* x, T* r) {
  const int d = rb.n * rb.m;
  const int nbp = 3 * rb.n * rb.nb;
  const bool nbb = needs_backbone(W, no);
  std::vector<T> U((size_t)Tn * d), bb(nbb ? (size_t)Tn * nbp : 0);
  for (int a = 0; a < d; ++a) U[a] = T(u_start[a]);
  for (int t = 1; t < Tn; ++t)
    for (int a = 0; a < d; ++a) U[(size_t)t * d + a] = x[(size_t)(t - 1) * d + a];
  std::vector<FkOut<T>> fk(Tn);
  for (int t = 0; t < Tn; ++t)
    forward_kinematics(rb, P, &U[(size_t)t * d], fk[t], nbb ? &bb[(size_t)t * nbp] : nullptr);
  T sl = T(std::sqrt(W.w_len)), sv = T(std::sqrt(W.rho_v)), sa = T(std::sqrt(W.rho_a));
  int k = 0;
  for (int t = 1; t < Tn; ++t) {
    for (int a = 0; a < 3; ++a) r[k++] = sl * (fk[t].p[a] - fk[t - 1].p[a]);
    for (int q = 0; q < d; ++q) {
      T v = (U[(size_t)t * d + q] - U[(size_t)(t - 1) * d + q]) / T(W.dt);
      r[k++] = sv * hinge(v - T(W.vmax));
      r[k++] = sv * hinge(T(-W.vmax) - v);
    }
    k += state_constraint_rows(rb, W, no, obs, &U[(size_t)t * d], fk[t],
                               nbb ? &bb[(size_t)t * nbp] : (const T*)nullptr, r + k, (T*)nullptr);
    if (t >= 2) {
      for (int q = 0; q < d; ++q) {
        T acc = (U[(size_t)t * d + q] - T(2.0) * U[(size_t)(t - 1) * d + q] + U[(size_t)(t - 2) * d + q]) /
                T(W.dt * W.dt);
        r[k++] = sa * hinge(acc - T(W.amax));
        r[k++] = sa * hinge(T(-W.amax) - acc);
      }
    }
  }
  pose_residual(OR_IK6, W, goal, fk[Tn - 1].R, fk[Tn - 1].p, r + k);
  k += 6;
  return k;
}

static int traj_rows(const OrRobot& rb, const OrWeights& W, int no, int Tn) {
  const int d = rb.n * rb.m;
  return (Tn - 1) * (3 + 2 * d + state_constraint_count(rb, W, no)) + std::max(0, Tn - 2) * 2 * d + 6;
}

struct TrajProblem {
  const OrRobot* rb;
  const OrWeights* W;
  int no;
  const double* obs;
  const double* u_start;
  const double* goal;
  int Tn;
  int nx() const { return (Tn - 1) * rb->n * rb->m; }
  int rows() const { return traj_rows(*rb, *W, no, Tn); }
  double cost(const double* x) const {
    std::vector<double> r(rows());
    Params<double> P = params_of<double>(*rb);
    traj_residual(*rb, P, *W, no, obs, u_start, goal, Tn, x, r.data());
    return half_sq(r.data(), rows());
  }
  // gradient of F by complex step on F itself
  void grad(const double* x, double* g) const {
    int n = nx();
    std::vector<cd> xc(n), r(rows());
    Params<cd> P = params_of<cd>(*rb);
    for (int c = 0; c < n; ++c) {
      for (int q = 0; q < n; ++q) xc[q] = cd(x[q], q == c ? CS_H : 0.0);
      traj_residual(*rb, P, *W, no, obs, u_start, goal, Tn, xc.data(), r.data());
      g[c] = half_sq(r.data(), rows()).imag() / CS_H;
    }
  }
};

// Projected-gradient refinement of a trajectory: pg_rule with the norm taken over all free states
// and the projection applied to every state's segments.
static void traj_pg(const TrajProblem& tp, double* x, int steps, double alpha0, double* F_out) {
  const OrRobot& rb = *tp.rb;
  const int d = rb.n * rb.m, Tn = tp.Tn;
  pg_rule(tp.nx(), x, steps, alpha0, [&tp](const double* xx) { return tp.cost(xx); },
          [&tp](const double* xx, double* g) { tp.grad(xx, g); },
          [&rb, d, Tn](const double* v, double* x1) {
            for (int t = 0; t < Tn - 1; ++t)
              for (int i = 0; i < rb.n; ++i)
                project_segment(&v[(size_t)t * d + rb.m * i], rb.m, rb.umax[i], &x1[(size_t)t * d + rb.m * i]);
          },
          F_out, nullptr);
}

// ---------------------------------------------------------------------------------------------
// Path following
// ---------------------------------------------------------------------------------------------

// Rows of one waypoint t against its reference pose: the IK residual (pose + state rows).
// The path residual stacks the waypoint rows for t = 0..H-1, then the smoothness rows
// sqrt(w_s)(u_t - u_{t-1}) for t = 1..H-1 (d each).
template <class T>
static int path_residual(const OrRobot& rb, const Params<T>& P, const OrWeights& W, int no,
                         const double* obs, const double* wp, int H, const T* x, T* r) {
  const int d = rb.n * rb.m;
  int k = 0;
  for (int t = 0; t < H; ++t)
    k += ik_residual(rb, P, W, no, obs, OR_IK6, wp + 7 * t, x + (size_t)t * d, r + k, (T*)nullptr);
  T ss = T(std::sqrt(W.w_s));
  for (int t = 1; t < H; ++t)
    for (int q = 0; q < d; ++q) r[k++] = ss * (x[(size_t)t * d + q] - x[(size_t)(t - 1) * d + q]);
  return k;
}

static int path_rows(const OrRobot& rb, const OrWeights& W, int no, int H) {
  return H * ik_rows(rb, W, no) + (H - 1) * rb.n * rb.m;
}

struct PathProblem {
  const OrRobot* rb;
  const OrWeights* W;
  int no;
  const double* obs;
  const double* wp;
  int H;
  int d() const { return rb->n * rb->m; }
  int nx() const { return H * d(); }
  double cost(const double* x) const {
    std::vector<double> r(path_rows(*rb, *W, no, H));
    Params<double> P = params_of<double>(*rb);
    path_residual(*rb, P, *W, no, obs, wp, H, x, r.data());
    return half_sq(r.data(), (int)r.size());
  }
  // F, A = J^T J and g = J^T r. The waypoint rows of t depend only on u_t, so their Jacobian block
  // is taken by complex step over u_t alone; each smoothness row has entries +-sqrt(w_s).
  double normal(const double* x, double* A, double* g) const {
    const int dd = d(), n = nx();
    for (size_t a = 0; a < (size_t)n * n; ++a) A[a] = 0.0;
    for (int a = 0; a < n; ++a) g[a] = 0.0;
    double F = 0.0;
    for (int t = 0; t < H; ++t) {
      IkProblem pb{rb, W, no, obs, OR_IK6, wp + 7 * t};
      int nr = pb.rows();
      std::vector<double> r(nr), J((size_t)nr * dd);
      pb.res(x + (size_t)t * dd, r.data());
      cs_jacobian([&pb](const cd* xx, cd* rr) { pb.cres(xx, rr); }, dd, nr, x + (size_t)t * dd, J.data());
      for (int k = 0; k < nr; ++k) F += 0.5 * r[k] * r[k];
      for (int a = 0; a < dd; ++a) {
        double s = 0;
        for (int k = 0; k < nr; ++k) s += J[(size_t)k * dd + a] * r[k];
        g[t * dd + a] += s;
        for (int b = 0; b < dd; ++b) {
          double m = 0;
          for (int k = 0; k < nr; ++k) m += J[(size_t)k * dd + a] * J[(size_t)k * dd + b];
          A[(size_t)(t * dd + a) * n + t * dd + b] += m;
        }
      }
    }
    const double ss = std::sqrt(W->w_s);
    for (int t = 1; t < H; ++t)
      for (int q = 0; q < dd; ++q) {
        int i1 = t * dd + q, i0 = (t - 1) * dd + q;  // row = ss (x[i1] - x[i0])
        double r = ss * (x[i1] - x[i0]);
        F += 0.5 * r * r;
        g[i1] += ss * r;
        g[i0] -= ss * r;
        A[(size_t)i1 * n + i1] += ss * ss;
        A[(size_t)i0 * n + i0] += ss * ss;
        A[(size_t)i1 * n + i0] -= ss * ss;
        A[(size_t)i0 * n + i1] -= ss * ss;
      }
    return F;
  }
};

// ---------------------------------------------------------------------------------------------
// Calibration: r(theta) = p(u_k; L, r_c) - p_k, k < K, theta = (L_1..n, r_c,1..n)
// ---------------------------------------------------------------------------------------------
template <class T>
static void calib_residual(const OrRobot& rb, const double* U, const double* Pm, int K, const T* theta, T* r) {
  const int d = rb.n * rb.m;
  Params<T> P;
  for (int i = 0; i < rb.n; ++i) { P.L[i] = theta[i]; P.rc[i] = theta[rb.n + i]; }
  std::vector<T> u(d);
  for (int k = 0; k < K; ++k) {
    for (int a = 0; a < d; ++a) u[a] = T(U[(size_t)k * d + a]);
    FkOut<T> o;
    forward_kinematics(rb, P, u.data(), o, (T*)nullptr);
    for (int a = 0; a < 3; ++a) r[3 * k + a] = o.p[a] - T(Pm[3 * k + a]);
  }
}

extern "C" {

int orc_traj_rows(const OrRobot* rb, const OrWeights* W, int no, int Tn) { return traj_rows(*rb, *W, no, Tn); }

// Trajectory cost / gradient / residuals of P problems. u_start [P][d], goal [P][7], obs
// [P][no][OR_OBS] (per problem), x [P][(Tn-1)][d] (the free states u_1..u_{Tn-1}).
int orc_traj_eval(const OrRobot* rb, const OrWeights* W, int no, const double* obs,
                  const double* u_start, const double* goal, int Tn, const double* x, int64_t P,
                  double* F, double* g, double* r, int threads) {
  if (Tn < 2) return 1;
  const int d = rb->n * rb->m;
  parallel_for(P, threads, [&](int64_t q) {
    TrajProblem tp{rb, W, no, no > 0 ? obs + (size_t)OR_OBS * no * q : nullptr, u_start + (size_t)d * q,
                   goal + 7 * q, Tn};
    const double* xq = x + (size_t)tp.nx() * q;
    if (F) F[q] = tp.cost(xq);
    if (g) tp.grad(xq, g + (size_t)tp.nx() * q);
    if (r) {
      Params<double> Pd = params_of<double>(*rb);
      traj_residual(*rb, Pd, *W, no, tp.obs, tp.u_start, tp.goal, Tn, xq, r + (size_t)tp.rows() * q);
    }
  });
  return 0;
}

int orc_traj_pg(const OrRobot* rb, const OrWeights* W, int no, const double* obs, const double* u_start,
                const double* goal, int Tn, double* x, int64_t P, int steps, double alpha0, double* F, int threads) {
  const int d = rb->n * rb->m;
  parallel_for(P, threads, [&](int64_t q) {
    TrajProblem tp{rb, W, no, no > 0 ? obs + (size_t)OR_OBS * no * q : nullptr, u_start + (size_t)d * q,
                   goal + 7 * q, Tn};
    traj_pg(tp, x + (size_t)tp.nx() * q, steps, alpha0, F + q);
  });
  return 0;
}

// Refinement and metrics of one trajectory from its initial states X [Tn][d] (X[0] = u_start):
// k_traj projected-gradient steps of the free states, then F, goal_pos / goal_rot, speed / accel
// (the largest |du|/dt / v_max and |d2u|/dt^2 / a_max) and lim_ok / col_ok (every state within
// limits / collision-free).
static void traj_refine_one(const OrRobot* rb, const OrWeights* W, int no, const double* sp, const double* u0,
                            const double* goal, int Tn, double* X, int k_traj, double alpha0, double lim_tol,
                            double* F, double* goal_pos, double* goal_rot, double* speed, double* accel,
                            uint8_t* lim_ok, uint8_t* col_ok) {
  const int d = rb->n * rb->m;
  TrajProblem tp{rb, W, no, sp, u0, goal, Tn};
  traj_pg(tp, X + d, k_traj, alpha0, F);
  double pos, rot;
  uint8_t lo, co;
  accept_one(*rb, no, sp, OR_IK6, goal, X + (size_t)(Tn - 1) * d, lim_tol, &pos, &rot, &lo, &co, W->rho_s > 0.0);
  *goal_pos = pos;
  *goal_rot = rot;
  bool lim = true, col = true;
  for (int t = 0; t < Tn; ++t) {
    double p2, r2;
    uint8_t l2, c2;
    accept_one(*rb, no, sp, OR_IK6, goal, X + (size_t)t * d, lim_tol, &p2, &r2, &l2, &c2, W->rho_s > 0.0);
    lim = lim && l2;
    col = col && c2;
  }
  double vm = 0, am = 0;
  for (int t = 1; t < Tn; ++t)
    for (int a = 0; a < d; ++a) {
      vm = std::max(vm, std::fabs(X[(size_t)t * d + a] - X[(size_t)(t - 1) * d + a]) / W->dt / W->vmax);
      if (t >= 2)
        am = std::max(am, std::fabs(X[(size_t)t * d + a] - 2 * X[(size_t)(t - 1) * d + a] + X[(size_t)(t - 2) * d + a]) /
                              (W->dt * W->dt) / W->amax);
    }
  *speed = vm;
  *accel = am;
  *lim_ok = lim;
  *col_ok = col;
}

// Trajectory planning per problem: IK to the goal pose (Algorithm 1 with ik_prm, seed counter p0 +
// q), linear interpolation u_t = u_start + (t / (Tn-1)) (u_goal - u_start), then k_traj
// projected-gradient steps. x_out [P][Tn][d] (all states, u_0 included); F_out [P]; goal_pos /
// goal_rot [P]; speed / accel [P]: the largest |du|/dt / v_max and |d2u|/dt^2 / a_max; lim_ok /
// col_ok [P]: every state within limits / collision-free.
int orc_solve_traj(const OrRobot* rb, const OrWeights* W, int no, const double* obs,
                   const double* u_start, const double* goal, int64_t P, int Tn, const OrIkParams* ik_prm,
                   int k_traj, double alpha0, double* x_out, double* F_out, double* goal_pos, double* goal_rot,
                   double* speed, double* accel, uint8_t* lim_ok, uint8_t* col_ok, int threads) {
  const int d = rb->n * rb->m;
  parallel_for(P, threads, [&](int64_t q) {
    const double* sp = no > 0 ? obs + (size_t)OR_OBS * no * q : nullptr;
    OrIkParams prm = *ik_prm;
    prm.p0 = ik_prm->p0 + q;
    double ug[OR_MAXSEG * 3], Fg, pe, re;
    uint8_t ok;
    orc_solve_ik(rb, W, no, sp, OR_IK6, goal + 7 * q, 1, &prm, ug, &Fg, &pe, &re, &ok, nullptr, nullptr, 1);
    double* X = x_out + (size_t)Tn * d * q;
    const double* u0 = u_start + (size_t)d * q;
    for (int t = 0; t < Tn; ++t)
      for (int a = 0; a < d; ++a) X[(size_t)t * d + a] = u0[a] + (double)t / (Tn - 1) * (ug[a] - u0[a]);
    traj_refine_one(rb, W, no, sp, u0, goal + 7 * q, Tn, X, k_traj, alpha0, ik_prm->lim_tol, F_out + q,
                    goal_pos + q, goal_rot + q, speed + q, accel + q, lim_ok + q, col_ok + q);
  });
  return 0;
}

// Trajectory refinement from given initial states (x_io [P][Tn][d] in, refined states out), with
// the metrics of orc_solve_traj: the second stage of Algorithm 2 after any initialiser.
int orc_traj_refine(const OrRobot* rb, const OrWeights* W, int no, const double* obs, const double* u_start,
                    const double* goal, int64_t P, int Tn, int k_traj, double alpha0, double lim_tol, double* x_io,
                    double* F_out, double* goal_pos, double* goal_rot, double* speed, double* accel,
                    uint8_t* lim_ok, uint8_t* col_ok, int threads) {
  const int d = rb->n * rb->m;
  parallel_for(P, threads, [&](int64_t q) {
    const double* sp = no > 0 ? obs + (size_t)OR_OBS * no * q : nullptr;
    traj_refine_one(rb, W, no, sp, u_start + (size_t)d * q, goal + 7 * q, Tn, x_io + (size_t)Tn * d * q, k_traj,
                    alpha0, lim_tol, F_out + q, goal_pos + q, goal_rot + q, speed + q, accel + q, lim_ok + q,
                    col_ok + q);
  });
  return 0;
}

// Calibration by LM on theta = (L, r_c): U [K][d] known displacements, Pm [K][3] measured tip
// positions. theta [2n] in/out (initial guess in), hist [iters][2n] nullable, F_out = final cost.
int orc_calibrate(const OrRobot* rb, const double* U, const double* Pm, int K, double* theta, int iters,
                  double lambda0, double* F_out, double* hist) {
  const int np = 2 * rb->n, nr = 3 * K;
  auto fr = [&](const double* th, double* r) { calib_residual(*rb, U, Pm, K, th, r); };
  auto fc = [&](const cd* th, cd* r) { calib_residual(*rb, U, Pm, K, th, r); };
  LmState st{lambda0, 2.0, 0.0};
  for (int it = 0; it < iters; ++it) {
    lm_iteration(fr, fc, np, nr, theta, st);
    if (hist) std::memcpy(hist + (size_t)it * np, theta, sizeof(double) * np);
  }
  std::vector<double> r(nr);
  fr(theta, r.data());
  *F_out = half_sq(r.data(), nr);
  return 0;
}

// The calibration residual r [3K] at theta (pose k's tip position minus its measurement).
int orc_calib_residual(const OrRobot* rb, const double* U, const double* Pm, int K, const double* theta, double* r) {
  calib_residual(*rb, U, Pm, K, theta, r);
  return 0;
}

// Jacobian of the calibration residual [3K][2n] by complex step (for the covariance pin).
int orc_calib_jacobian(const OrRobot* rb, const double* U, const double* Pm, int K, const double* theta, double* J) {
  auto fc = [&](const cd* th, cd* r) { calib_residual(*rb, U, Pm, K, th, r); };
  cs_jacobian(fc, 2 * rb->n, 3 * K, theta, J);
  return 0;
}

int orc_path_rows(const OrRobot* rb, const OrWeights* W, int no, int H) { return path_rows(*rb, *W, no, H); }

// Path residual r [rows] of one path (obs [no][OR_OBS], waypoints wp [H][7], x [H][d]); and its full
// Jacobian J [rows][H d] by complex step over all H d variables (small H; pins the blockwise
// assembly of the normal equations).
int orc_path_residual(const OrRobot* rb, const OrWeights* W, int no, const double* obs, const double* wp,
                      int H, const double* x, double* r, double* J) {
  Params<double> Pd = params_of<double>(*rb);
  path_residual(*rb, Pd, *W, no, obs, wp, H, x, r);
  if (J) {
    const int n = H * rb->n * rb->m, nr = path_rows(*rb, *W, no, H);
    cs_jacobian([&](const cd* xx, cd* rr) {
      Params<cd> P = params_of<cd>(*rb);
      path_residual(*rb, P, *W, no, obs, wp, H, xx, rr);
    }, n, nr, x, J);
  }
  return 0;
}

// Joint LM on one path: x [H][d] in/out, iters iterations; hist [iters][H][d] nullable.
// trace [iters][2] (nullable): the cost at each iteration's start and at its trial point.
int orc_path_lm(const OrRobot* rb, const OrWeights* W, int no, const double* obs, const double* wp, int H,
                double* x, int iters, double* lam, double* nu, double* F_out, double* hist, uint8_t* acc,
                double* trace) {
  PathProblem pp{rb, W, no, obs, wp, H};
  LmState st{*lam, *nu, 0.0};
  const int n = pp.nx();
  for (int it = 0; it < iters; ++it) {
    int a = lm_iteration_ag([&](const double* xx, double* A, double* g) { return pp.normal(xx, A, g); },
                            [&](const double* xx) { return pp.cost(xx); }, n, x, st);
    if (acc) acc[it] = (uint8_t)a;
    if (hist) std::memcpy(hist + (size_t)it * n, x, sizeof(double) * n);
    if (trace) { trace[2 * it] = st.Fstart; trace[2 * it + 1] = st.Ftrial; }
  }
  *lam = st.lambda;
  *nu = st.nu;
  *F_out = pp.cost(x);
  return 0;
}

// Path following per path: IK at waypoint 0 (Algorithm 1 with ik_prm, seed counter p0 + q), then
// for t >= 1 k_warm LM iterations of the waypoint's IK residual from u*_{t-1}, then k_joint joint
// LM iterations over the whole path (lambda0 = ik_prm->lambda0). obs [P][no][OR_OBS], wp [P][H][7].
// Outputs x_out [P][H][d], F_out [P] (joint cost), pos / rot [P][H] (per-waypoint errors),
// stage_x [P][H][d] (nullable: the trajectory before the joint stage), lim_ok / col_ok [P];
// trace [P][(H-1) k_warm + k_joint][2] (nullable): start and trial costs of every LM iteration of the
// warm sweep (waypoint by waypoint) and then of the joint stage.
int orc_solve_path(const OrRobot* rb, const OrWeights* W, int no, const double* obs, const double* wp,
                   int64_t P, int H, const OrIkParams* ik_prm, int k_warm, int k_joint, double* x_out,
                   double* F_out, double* pos, double* rot, double* stage_x, uint8_t* lim_ok, uint8_t* col_ok,
                   double* trace, int threads) {
  const int d = rb->n * rb->m;
  parallel_for(P, threads, [&](int64_t q) {
    const double* sp = no > 0 ? obs + (size_t)OR_OBS * no * q : nullptr;
    const double* wq = wp + (size_t)7 * H * q;
    double* X = x_out + (size_t)H * d * q;
    double* tr = trace ? trace + 2 * ((size_t)(H - 1) * k_warm + k_joint) * q : nullptr;
    OrIkParams prm = *ik_prm;
    prm.p0 = ik_prm->p0 + q;
    double Fg, pe, re;
    uint8_t ok;
    orc_solve_ik(rb, W, no, sp, OR_IK6, wq, 1, &prm, X, &Fg, &pe, &re, &ok, nullptr, nullptr, 1);
    for (int t = 1; t < H; ++t) {
      double* xt = X + (size_t)t * d;
      std::memcpy(xt, X + (size_t)(t - 1) * d, sizeof(double) * d);
      IkProblem pb{rb, W, no, sp, OR_IK6, wq + 7 * t};
      LmState st{ik_prm->lambda0, 2.0, 0.0};
      for (int it = 0; it < k_warm; ++it) {
        lm_iteration([&pb](const double* xx, double* rr) { pb.res(xx, rr); },
                     [&pb](const cd* xx, cd* rr) { pb.cres(xx, rr); }, d, pb.rows(), xt, st);
        if (tr) { tr[2 * ((t - 1) * k_warm + it)] = st.Fstart; tr[2 * ((t - 1) * k_warm + it) + 1] = st.Ftrial; }
      }
    }
    if (stage_x) std::memcpy(stage_x + (size_t)H * d * q, X, sizeof(double) * H * d);
    double lam = ik_prm->lambda0, nu = 2.0;
    orc_path_lm(rb, W, no, sp, wq, H, X, k_joint, &lam, &nu, &F_out[q], nullptr, nullptr,
                tr ? tr + 2 * (size_t)(H - 1) * k_warm : nullptr);
    bool lim = true, col = true;
    for (int t = 0; t < H; ++t) {
      uint8_t lo, co;
      accept_one(*rb, no, sp, OR_IK6, wq + 7 * t, X + (size_t)t * d, ik_prm->lim_tol, &pos[(size_t)H * q + t],
                 &rot[(size_t)H * q + t], &lo, &co, W->rho_s > 0.0);
      lim = lim && lo;
      col = col && co;
    }
    lim_ok[q] = lim;
    col_ok[q] = col;
  });
  return 0;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// PRM exploration of Algorithm 2 (Sec. IV-B, "Trajectory Planning"): ParallelSample,
// ParallelConnect, ConnectToRoadmap, Dijkstra and ResampleLinear, written out plainly. Readings:
//  * ParallelSample: node i of roadmap r is the first of `attempts` hexagon-uniform draws (the
//    SampleSeeds generator with problem r, seed i, attempt a) whose backbone is collision-free;
//    a node with no such draw is invalid and takes no part in the graph.
//  * ParallelConnect: the k nearest valid nodes of every valid node (squared Euclidean distance in
//    u, ties to the lower index); the edge {i, j} exists when i lists j or j lists i and the
//    straight segment is collision-free at n_check interior states x_a + c/(n_check+1) (x_b - x_a),
//    c = 1..n_check, interpolated from the lower index a to the higher b. Weight: the Euclidean
//    distance, the squared distance summed in coordinate order.
//  * ConnectToRoadmap: the start (goal) state is linked to those of its k nearest valid nodes whose
//    segment from the state to the node is collision-free at the n_check interior states; there
//    is no direct start-goal edge.
//  * Dijkstra from the start; the path is read back from the goal through the predecessor of the
//    lowest index among the neighbours u with d(u) < d(v) and d(u) + w(u, v) == d(v) (start =
//    index N, goal = index N + 1), which makes it unique when several paths tie.
//  * ResampleLinear: T states at equal arc length along the path (arc length = the Dijkstra
//    distances), state 0 the start and state T-1 the goal; with no path, the linear interpolation
//    u_start + t/(T-1) (u_goal - u_start).
// The PRM functions take sphere obstacles only, as [no][4] = (centre, radius).
// ---------------------------------------------------------------------------------------------

static bool prm_collides(const OrRobot& rb, const Params<double>& Pd, double delta, int no, const double* sp,
                         const double* x) {
  if (no == 0) return false;
  FkOut<double> o;
  std::vector<double> bb(3 * rb.n * rb.nb);
  forward_kinematics(rb, Pd, x, o, bb.data());
  for (int k = 0; k < rb.n * rb.nb; ++k)
    for (int c = 0; c < no; ++c) {
      const double* s = sp + 4 * c;
      const double dx = bb[3 * k] - s[0], dy = bb[3 * k + 1] - s[1], dz = bb[3 * k + 2] - s[2];
      const double reach = s[3] + rb.rbody + delta;
      if (dx * dx + dy * dy + dz * dz < reach * reach) return true;
    }
  return false;
}

static double prm_dist2(const double* a, const double* b, int d) {
  double s = 0.0;
  for (int q = 0; q < d; ++q) {
    const double t = a[q] - b[q];
    s = s + t * t;
  }
  return s;
}

// Is the segment from xa to xb free at its n_check interior states?
static bool prm_segment_free(const OrRobot& rb, const Params<double>& Pd, double delta, int no, const double* sp,
                             const double* xa, const double* xb, int n_check) {
  const int d = rb.n * rb.m;
  double x[OR_MAXSEG * 3];
  for (int c = 1; c <= n_check; ++c) {
    const double s = (double)c / (double)(n_check + 1);
    for (int q = 0; q < d; ++q) x[q] = xa[q] + s * (xb[q] - xa[q]);
    if (prm_collides(rb, Pd, delta, no, sp, x)) return false;
  }
  return true;
}

// The k nearest valid nodes of state x (excluding node `self`), ascending by (distance^2, index).
static std::vector<std::pair<double, int>> prm_nearest(const double* nodes, const uint8_t* ok, int N, int d,
                                                       const double* x, int self, int k) {
  std::vector<std::pair<double, int>> c;
  for (int j = 0; j < N; ++j)
    if (ok[j] && j != self) c.push_back({prm_dist2(x, nodes + (size_t)j * d, d), j});
  std::sort(c.begin(), c.end());
  if ((int)c.size() > k) c.resize(k);
  return c;
}

extern "C" {

// ParallelSample for roadmap r: nodes [N][d], ok [N].
int orc_prm_sample(const OrRobot* rb, double delta, int no, const double* spheres, uint64_t key, int64_t r, int N,
                   int attempts, double* nodes, uint8_t* ok) {
  const int d = rb->n * rb->m;
  Params<double> Pd = params_of<double>(*rb);
  for (int i = 0; i < N; ++i) {
    double* x = nodes + (size_t)i * d;
    ok[i] = 0;
    for (int a = 0; a < attempts && !ok[i]; ++a) {
      for (int s = 0; s < rb->n; ++s) {
        double U[3];
        for (int w = 0; w < 3; ++w) U[w] = u01_from(splitmix64_at(key, seed_counter(r, i, a, s, w)));
        hexagon_point(rb->umax[s], U[0], U[1], U[2], x + 3 * s);
      }
      ok[i] = !prm_collides(*rb, Pd, delta, no, spheres, x);
    }
  }
  return 0;
}

// k nearest valid neighbours of every valid node: nbr [N][k], -1 where there are fewer (and for
// invalid nodes).
int orc_prm_knn(const double* nodes, const uint8_t* ok, int N, int d, int k, int32_t* nbr) {
  for (int i = 0; i < N; ++i) {
    for (int c = 0; c < k; ++c) nbr[(size_t)i * k + c] = -1;
    if (!ok[i]) continue;
    std::vector<std::pair<double, int>> c = prm_nearest(nodes, ok, N, d, nodes + (size_t)i * d, i, k);
    for (size_t e = 0; e < c.size(); ++e) nbr[(size_t)i * k + e] = c[e].second;
  }
  return 0;
}

// Is the segment from xa to xb collision-free at its n_check interior states? (1 / 0)
int orc_prm_segment_free(const OrRobot* rb, double delta, int no, const double* spheres, const double* xa,
                         const double* xb, int n_check) {
  Params<double> Pd = params_of<double>(*rb);
  return prm_segment_free(*rb, Pd, delta, no, spheres, xa, xb, n_check) ? 1 : 0;
}

// ParallelConnect: the roadmap graph in CSR form, rows in node order, columns ascending:
// row [N+1], col [2 N k] and wt [2 N k] (capacity), from nodes, ok and the kNN lists nbr.
int orc_prm_connect(const OrRobot* rb, double delta, int no, const double* spheres, const double* nodes,
                    const uint8_t* ok, const int32_t* nbr, int N, int k, int n_check, int32_t* row, int32_t* col,
                    double* wt) {
  const int d = rb->n * rb->m;
  Params<double> Pd = params_of<double>(*rb);
  std::vector<std::vector<uint8_t>> adj(N, std::vector<uint8_t>(N, 0));
  for (int i = 0; i < N; ++i)
    for (int c = 0; c < k && ok[i]; ++c) {  // an invalid node lists no neighbours
      const int j = nbr[(size_t)i * k + c];
      if (j < 0 || adj[i][j]) continue;
      const int a = std::min(i, j), b = std::max(i, j);
      if (prm_segment_free(*rb, Pd, delta, no, spheres, nodes + (size_t)a * d, nodes + (size_t)b * d, n_check))
        adj[i][j] = adj[j][i] = 1;
    }
  int e = 0;
  for (int i = 0; i < N; ++i) {
    row[i] = e;
    for (int j = 0; j < N; ++j)
      if (adj[i][j]) {
        col[e] = j;
        wt[e] = std::sqrt(prm_dist2(nodes + (size_t)i * d, nodes + (size_t)j * d, d));
        ++e;
      }
  }
  row[N] = e;
  return 0;
}

// One query on a roadmap (nodes [N][d], ok, CSR row/col/wt): ConnectToRoadmap of u_start and
// u_goal, Dijkstra, ResampleLinear to X [T][d]. Returns the path length (the distance of the
// goal, +inf with no path) in *length and the number of path edges (0 with no path) in *hops;
// path [N + 2] (nullable) receives the path's vertex indices from the start.
int orc_prm_query(const OrRobot* rb, double delta, int no, const double* spheres, const double* nodes,
                  const uint8_t* ok, const int32_t* row, const int32_t* col, const double* wt, int N, int k,
                  int n_check, const double* us, const double* ug, int T, double* X, double* length, int32_t* hops,
                  int32_t* path) {
  const int d = rb->n * rb->m;
  Params<double> Pd = params_of<double>(*rb);
  const int S = N, G = N + 1, V = N + 2;
  // adjacency lists of the query graph: roadmap edges plus the start and goal links
  std::vector<std::vector<std::pair<int, double>>> nb(V);
  for (int i = 0; i < N; ++i)
    for (int e = row[i]; e < row[i + 1]; ++e) nb[i].push_back({col[e], wt[e]});
  const double* q[2] = {us, ug};
  for (int side = 0; side < 2; ++side) {
    const int vq = side == 0 ? S : G;
    for (auto& c : prm_nearest(nodes, ok, N, d, q[side], -1, k))
      if (prm_segment_free(*rb, Pd, delta, no, spheres, q[side], nodes + (size_t)c.second * d, n_check)) {
        const double w = std::sqrt(c.first);
        nb[vq].push_back({c.second, w});
        nb[c.second].push_back({vq, w});
      }
  }
  // Dijkstra (binary heap, lazy deletion)
  std::vector<double> dist(V, INFINITY);
  std::vector<uint8_t> done(V, 0);
  std::priority_queue<std::pair<double, int>, std::vector<std::pair<double, int>>, std::greater<>> pq;
  dist[S] = 0.0;
  pq.push({0.0, S});
  while (!pq.empty()) {
    const auto [du, u] = pq.top();
    pq.pop();
    if (done[u]) continue;
    done[u] = 1;
    for (auto& [v, w] : nb[u])
      if (du + w < dist[v]) {
        dist[v] = du + w;
        pq.push({dist[v], v});
      }
  }
  *length = dist[G];
  auto xv = [&](int v) { return v == S ? us : (v == G ? ug : nodes + (size_t)v * d); };
  if (!(dist[G] < INFINITY)) {
    *hops = 0;
    for (int t = 0; t < T; ++t)
      for (int a = 0; a < d; ++a) X[(size_t)t * d + a] = us[a] + (double)t / (T - 1) * (ug[a] - us[a]);
    return 0;
  }
  // path from the goal back to the start through the canonical predecessors
  std::vector<int> pth{G};
  for (int v = G; v != S && (int)pth.size() <= V;) {
    int best = -1;
    for (auto& [u, w] : nb[v])
      if (dist[u] < dist[v] && dist[u] + w == dist[v] && (best < 0 || u < best)) best = u;
    v = best;
    pth.push_back(v);
  }
  std::reverse(pth.begin(), pth.end());
  const int M = (int)pth.size() - 1;
  *hops = M;
  if (path)
    for (int j = 0; j <= M; ++j) path[j] = pth[j];
  // ResampleLinear
  const double Lt = dist[G];
  for (int t = 0; t < T; ++t) {
    double* x = X + (size_t)t * d;
    if (t == 0 || t == T - 1) {
      std::memcpy(x, t == 0 ? us : ug, sizeof(double) * d);
      continue;
    }
    const double s = (double)t / (double)(T - 1) * Lt;
    int j = 0;
    while (j + 1 < M && dist[pth[j + 1]] <= s) ++j;
    const double lam = (s - dist[pth[j]]) / (dist[pth[j + 1]] - dist[pth[j]]);
    const double *xa = xv(pth[j]), *xb = xv(pth[j + 1]);
    for (int a = 0; a < d; ++a) x[a] = xa[a] + lam * (xb[a] - xa[a]);
  }
  return 0;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Self-contact rows on their own (the rows of self_rows_bb above, from the state's backbone).
// ---------------------------------------------------------------------------------------------
template <class T>
static int self_rows(const OrRobot& rb, const Params<T>& P, const T* u, double rho_s, double delta, T* r) {
  FkOut<T> fk;
  std::vector<T> bb(3 * rb.n * rb.nb);
  forward_kinematics(rb, P, u, fk, bb.data());
  return self_rows_bb(rb, bb.data(), rho_s, delta, r, (T*)nullptr);
}

extern "C" {

int orc_self_row_count(const OrRobot* rb) { return self_row_count(*rb); }

// Self-contact rows r [B][rows] and cost F [B] of states u [B][d]; with g (nullable) also the
// complex-step gradient dF/du [B][d].
int orc_self_rows(const OrRobot* rb, double rho_s, double delta, const double* u, int64_t B, double* r, double* F,
                  double* g) {
  const int d = rb->n * rb->m, nr = self_row_count(*rb);
  Params<double> P = params_of<double>(*rb);
  Params<cd> Pc = params_of<cd>(*rb);
  std::vector<cd> rc(nr > 0 ? nr : 1), uc(d);
  for (int64_t b = 0; b < B; ++b) {
    const double* x = u + (size_t)d * b;
    double* rr = r + (size_t)nr * b;
    self_rows(*rb, P, x, rho_s, delta, rr);
    double f = 0.0;
    for (int k = 0; k < nr; ++k) f += 0.5 * rr[k] * rr[k];
    F[b] = f;
    if (!g) continue;
    const double h = 1e-30;
    for (int q = 0; q < d; ++q) {
      for (int a = 0; a < d; ++a) uc[a] = cd(x[a], a == q ? h : 0.0);
      self_rows(*rb, Pc, uc.data(), rho_s, delta, rc.data());
      cd fc(0.0);
      for (int k = 0; k < nr; ++k) fc += 0.5 * rc[k] * rc[k];
      g[(size_t)d * b + q] = fc.imag() / h;
    }
  }
  return 0;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Coupled tendon routing (Eq. l_eq read literally: tendon j of the robot runs through several
// segments and its length is the sum of the per-segment lengths of Eq. 4). Model B: the tendons
// that terminate at segment s run through segments 1..s at the angles alpha_j, so the actuator
// displacement of tendon j of segment s is the prefix sum q_sj = sum_{i <= s} u_ij of the
// per-segment displacements u_ij = l_ij - L_i used everywhere above (model A); conversely
// u_sj = q_sj - q_(s-1)j. Standalone, ahead of any solver that takes actuator displacements.
// ---------------------------------------------------------------------------------------------
extern "C" {

// u [B][n m] (model A) -> q [B][n m] (model B actuator displacements).
int orc_routing_b_from_a(const OrRobot* rb, const double* u, int64_t B, double* q) {
  const int n = rb->n, m = rb->m;
  for (int64_t b = 0; b < B; ++b)
    for (int j = 0; j < m; ++j) {
      double s = 0.0;
      for (int i = 0; i < n; ++i) {
        s = s + u[(size_t)b * n * m + i * m + j];
        q[(size_t)b * n * m + i * m + j] = s;
      }
    }
  return 0;
}

// Gradient in actuator coordinates: with u = D q (u_s = q_s - q_(s-1)), g_q = D^T g_u, i.e.
// g_q,sj = g_u,sj - g_u,(s+1)j (and g_u,nj for the last segment). g_u, g_q [B][n m].
int orc_routing_b_grad(const OrRobot* rb, const double* g_u, int64_t B, double* g_q) {
  const int n = rb->n, m = rb->m;
  for (int64_t b = 0; b < B; ++b)
    for (int j = 0; j < m; ++j)
      for (int i = 0; i < n; ++i) {
        const double* g = g_u + (size_t)b * n * m;
        g_q[(size_t)b * n * m + i * m + j] = i + 1 < n ? g[i * m + j] - g[(i + 1) * m + j] : g[i * m + j];
      }
  return 0;
}

// q [B][n m] (model B) -> u [B][n m] (model A).
int orc_routing_a_from_b(const OrRobot* rb, const double* q, int64_t B, double* u) {
  const int n = rb->n, m = rb->m;
  for (int64_t b = 0; b < B; ++b)
    for (int j = 0; j < m; ++j)
      for (int i = 0; i < n; ++i) {
        const double* qb = q + (size_t)b * n * m;
        u[(size_t)b * n * m + i * m + j] = i == 0 ? qb[j] : qb[i * m + j] - qb[(i - 1) * m + j];
      }
  return 0;
}

}  // extern "C"
