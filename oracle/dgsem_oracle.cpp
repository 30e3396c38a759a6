// Plain FP64 CPU oracle of the split-form DGSEM time derivative and its
// low-storage Runge-Kutta loop (GALAEXI, Sec. 3.1, Eqs. 1-3).
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
// reference that the CUDA path is checked against.  Only the test suite, the
// smoke entry and the benchmark's CPU-baseline leg may load it; the CUDA
// library never links, includes or calls it, and it shares no code with it.
//
// Everything is nested loops in the order of the mathematics; the scalar type
// is a template parameter so that the same code evaluates the tangent-linear
// operator with forward-mode dual numbers.
//
// Readings where the paper is silent (each listed in the design notes):
//  * p = (gamma-1) rho eps (the printed (1-gamma) is a sign typo, Sec. 3.1).
//  * LGL collocation, strong split form; curl-form metric terms (Kopriva 2006).
//  * Surface flux: local Lax-Friedrichs (or the two-point EC flux itself, or
//    Roe's flux with the Harten-Hyman entropy fix, the choice of Sec. 3.1);
//    viscous surface flux = arithmetic mean of both sides (BR1, Sec. 3.1).
//  * BR1 lifting of (u, v, w, T) with the non-conservative strong volume part.
//  * Two-point flux of Chandrashekar (2013) with the kinetic-energy term
//    1/2 * mean of |u|^2 (the form that satisfies Tadmor's condition).
//  * Logarithmic mean by the Ismail-Roe (2009) series/log split, with the
//    switch at xi^2 < 1e-4 and four series terms (truncation < 1e-17).
//  * Viscosity constant or by Sutherland's law mu0 (T/T_ref)^(3/2)
//    (T_ref + S)/(T + S) at each node's own temperature (the law the paper
//    names for its dissipation diagnostic, Sec. 4.2); Stokes hypothesis,
//    lambda = mu(T) c_p / Pr.
//  * Derivatives at the kinks of the LLF speed max(|u.n| + c) (ties, u.n = 0,
//    to within 1e-12 of the local scale) are the mean of the one-sided ones.
//  * LSERK4-5 of Carpenter and Kennedy (1994), or RK4-14 of Niegemann, Diehl
//    and Busch (2012), 2N storage.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include <algorithm>
#include <type_traits>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace orc {

// The element and face loops of the FP64 operator may run on several host
// threads when this file is built with OpenMP (the timed CPU baseline).  Each
// iteration writes only its own element's (or master face's) values and
// evaluates them with exactly the serial arithmetic, so the result is the
// serial result bit for bit.  The dual-number and counting scalars always run
// serially (the counter is a global).
template <class T> constexpr bool kParallel = std::is_same<T, double>::value;

// ---------------------------------------------------------------------------
// Forward-mode dual number (value, one tangent direction).
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double a) : v(a), d(0) {}
  Dual(double a, double b) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual& operator*=(Dual& a, Dual b) { a = a * b; return a; }
inline Dual sqrt(Dual a) { double s = std::sqrt(a.v); return Dual(s, a.d / (2.0 * s)); }
inline Dual log(Dual a) { return Dual(std::log(a.v), a.d / a.v); }
inline Dual fabs(Dual a) { return a.v < 0 ? -a : a; }     // branch follows the value
inline bool operator<(Dual a, Dual b) { return a.v < b.v; }
inline bool operator>(Dual a, Dual b) { return a.v > b.v; }
inline double val(Dual a) { return a.v; }
inline double val(double a) { return a; }
using std::sqrt; using std::log; using std::fabs;
// max with ties going to the first argument (the value decides the branch)
template <class T> inline T vmax(T a, T b) { return (val(b) > val(a)) ? b : a; }

// Operation-counting scalar: evaluates in double and counts each arithmetic
// operation that has a state-dependent operand (+ and - as additions, *, /,
// sqrt and log apart; a sign change is free).  Products of geometry or basis
// values alone stay in double and are not counted.  It serves only to count
// the floating-point work of the operator as this oracle states it.
struct OpCount { unsigned long long add = 0, mul = 0, div = 0, sqrt = 0, log = 0; };
static OpCount g_ops;
struct Counted {
  double v;
  Counted() : v(0) {}
  Counted(double a) : v(a) {}
};
inline Counted operator+(Counted a, Counted b) { ++g_ops.add; return Counted(a.v + b.v); }
inline Counted operator-(Counted a, Counted b) { ++g_ops.add; return Counted(a.v - b.v); }
inline Counted operator-(Counted a) { return Counted(-a.v); }
inline Counted operator*(Counted a, Counted b) { ++g_ops.mul; return Counted(a.v * b.v); }
inline Counted operator/(Counted a, Counted b) { ++g_ops.div; return Counted(a.v / b.v); }
inline Counted& operator+=(Counted& a, Counted b) { a = a + b; return a; }
inline Counted& operator-=(Counted& a, Counted b) { a = a - b; return a; }
inline Counted& operator*=(Counted& a, Counted b) { a = a * b; return a; }
inline Counted sqrt(Counted a) { ++g_ops.sqrt; return Counted(std::sqrt(a.v)); }
inline Counted log(Counted a) { ++g_ops.log; return Counted(std::log(a.v)); }
inline Counted fabs(Counted a) { return Counted(std::fabs(a.v)); }
inline bool operator<(Counted a, Counted b) { return a.v < b.v; }
inline bool operator>(Counted a, Counted b) { return a.v > b.v; }
inline double val(Counted a) { return a.v; }

// Non-differentiable points of the LLF speed max(|u.n| + c): where the two
// arguments tie, or u.n vanishes, to within 1e-12 of the local scale (as on
// the symmetry planes of a symmetric flow, where the values differ only by
// rounding), the derivative is the mean of the one-sided derivatives, which
// is what central differences measure there.  Elsewhere the value decides.
inline double vmax_kink(double a, double b) { return b > a ? b : a; }
inline Dual vmax_kink(Dual a, Dual b) {
  if (std::fabs(a.v - b.v) <= 1e-12 * std::max(std::fabs(a.v), std::fabs(b.v)))
    return Dual(b.v > a.v ? b.v : a.v, 0.5 * (a.d + b.d));
  return b.v > a.v ? b : a;
}
inline Counted vmax_kink(Counted a, Counted b) { return b.v > a.v ? b : a; }
inline double abs_kink(double x, double) { return std::fabs(x); }
inline Counted abs_kink(Counted x, double) { return Counted(std::fabs(x.v)); }
inline Dual abs_kink(Dual x, double scale) {
  if (std::fabs(x.v) <= 1e-12 * scale) return Dual(std::fabs(x.v), 0.0);
  return x.v < 0 ? -x : x;
}

// ---------------------------------------------------------------------------
// 1-D basis on Legendre-Gauss-Lobatto nodes (Sec. 3.1: collocation at LGL
// nodes).  Nodes: +-1 and the roots of P'_N, found by Newton's method on
// q = P_{N+1} - P_{N-1} (which is proportional to (1-x^2) P'_N).
static void legendre_q(int N, double x, double& q, double& dq, double& LN) {
  // Three-term recurrence for P_k and P'_k.
  double Lm2 = 1.0, Lm1 = x, dLm2 = 0.0, dLm1 = 1.0;
  double L = x, dL = 1.0;
  std::vector<double> Ls(N + 2), dLs(N + 2);
  Ls[0] = 1.0; dLs[0] = 0.0; Ls[1] = x; dLs[1] = 1.0;
  for (int k = 2; k <= N + 1; ++k) {
    L = ((2.0 * k - 1.0) * x * Lm1 - (k - 1.0) * Lm2) / k;
    dL = dLm2 + (2.0 * k - 1.0) * Lm1;
    Lm2 = Lm1; Lm1 = L; dLm2 = dLm1; dLm1 = dL;
    Ls[k] = L; dLs[k] = dL;
  }
  q = Ls[N + 1] - Ls[N - 1];
  dq = dLs[N + 1] - dLs[N - 1];
  LN = Ls[N];
}

struct Basis {
  int N, n;
  std::vector<double> x, w, D;   // D[i*n + j] = l_j'(x_i)
};

static Basis make_basis(int N) {
  Basis b; b.N = N; b.n = N + 1;
  int n = N + 1;
  b.x.assign(n, 0.0); b.w.assign(n, 0.0); b.D.assign(n * n, 0.0);
  b.x[0] = -1.0; b.x[N] = 1.0;
  for (int j = 1; j < N; ++j) {
    double xj = -std::cos(M_PI * j / N);   // Chebyshev-Gauss-Lobatto start
    for (int it = 0; it < 100; ++it) {
      double q, dq, LN;
      legendre_q(N, xj, q, dq, LN);
      double dx = -q / dq;
      xj += dx;
      if (std::fabs(dx) <= 1e-16 * std::fabs(xj)) break;
    }
    b.x[j] = xj;
  }
  // exact symmetry about 0
  for (int j = 0; j < n / 2; ++j) {
    double m = 0.5 * (b.x[N - j] - b.x[j]);
    b.x[j] = -m; b.x[N - j] = m;
  }
  if (N % 2 == 0) b.x[N / 2] = 0.0;
  for (int j = 0; j < n; ++j) {
    double q, dq, LN;
    legendre_q(N, b.x[j], q, dq, LN);
    b.w[j] = 2.0 / (N * (N + 1.0) * LN * LN);
  }
  // Differentiation matrix from barycentric weights; diagonal by the
  // negative-sum rule so that D applied to a constant is exactly zero.
  std::vector<double> lam(n, 1.0);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k)
      if (k != j) lam[j] /= (b.x[j] - b.x[k]);
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      double d = (lam[j] / lam[i]) / (b.x[i] - b.x[j]);
      b.D[i * n + j] = d;
      s += d;
    }
    b.D[i * n + i] = -s;
  }
  return b;
}

// Lagrange interpolation matrix from ngeo+1 equispaced points on [-1,1] to
// the LGL nodes: V[i*(ngeo+1) + k] = l_k(x_i).
static std::vector<double> equi_to_lgl(int ngeo, const Basis& b) {
  int m = ngeo + 1;
  std::vector<double> eta(m), V(b.n * m);
  for (int k = 0; k < m; ++k) eta[k] = -1.0 + 2.0 * k / ngeo;
  for (int i = 0; i < b.n; ++i)
    for (int k = 0; k < m; ++k) {
      double l = 1.0;
      for (int j = 0; j < m; ++j)
        if (j != k) l *= (b.x[i] - eta[j]) / (eta[k] - eta[j]);
      V[i * m + k] = l;
    }
  return V;
}

// ---------------------------------------------------------------------------
struct Params {
  double gamma, R, Pr, mu;
  int surf_flux;   // 0: local Lax-Friedrichs, 1: entropy-conservative two-point flux, 2: Roe + Harten-Hyman
  int source;      // 0: none, 1: density-wave manufactured solution
  double mms_amp;
  int vol_flux;    // 0: Chandrashekar EC/KEP two-point flux; 1: arithmetic mean of
                   //    the Euler flux (a test variant equal to the standard DGSEM)
  int visc_law;    // 0: constant mu; 1: Sutherland's law
  double T_ref, S_suth;   // Sutherland reference temperature and constant
};

// Legendre-Gauss basis (the alternative node set of Sec. 3.1): the N+1 roots
// of P_{N+1}, quadrature weights, collocation derivative, the Lagrange basis at
// the interval ends, and the LGL basis evaluated at the Gauss nodes (geometry).
struct GaussBasis {
  int N, n;
  std::vector<double> x, w, D;   // D[i*n + j] = l_j'(x_i)
  std::vector<double> lm, lp;    // l_j(-1), l_j(+1)
  std::vector<double> VL;        // VL[i*n + j] = l^LGL_j(x_i)
};

struct Ctx {
  int N, n, P, E;
  int nodes;                  // 0: LGL (split form), 1: Legendre-Gauss (standard weak form)
  int rk;                     // 0: LSERK4-5, 1: RK4-14
  Params prm;
  Basis b;
  GaussBasis g;
  std::vector<double> X;      // [e][c][P]
  std::vector<double> Ja;     // [e][d][l][P]  contravariant metric J a^d, component l
  std::vector<double> J;      // [e][P]
  std::vector<int> nbr;       // [e][6][3]
  std::vector<int> face_id;   // [e][6]
  std::vector<int> master;    // [e][6] 1 if (e,f) is the master side
  int nfaces;
  std::vector<double> fn;     // [face][3][n*n]  unit normal of the master side
  std::vector<double> fsJ;    // [face][n*n]     surface element of the master side
  mutable std::vector<int> fv_mask;   // [e] 1: FV sub-cell element (empty: none)
  // automatic DG/FV switching before every evaluation of R(U): the Persson
  // indicator of the evaluated state against two log10 thresholds
  bool sw_on = false;
  int sw_var = 2;
  double sw_up = 0.0, sw_low = 0.0;
  mutable double sw_margin = 1e300;   // smallest |log10 eta - threshold| met (test hook)
  // mortars (non-conforming faces, 2:1): [m][14] = big (e, f), four small (e, f, flip)
  int M = 0;
  std::vector<int> mortars;
  std::vector<double> mI;     // [2][n][n]: l_j at the nodes of half k of [-1, 1] (interpolation)
  std::string err;
};

static inline int vidx(int n, int i, int j, int k) { return i + n * (j + n * k); }

// Volume node of face node (p,q) of local face f = 2d + s.
static inline int face_vol(int n, int f, int p, int q) {
  int d = f / 2, s = f % 2, N = n - 1;
  int e = s * N;
  if (d == 0) return vidx(n, e, p, q);
  if (d == 1) return vidx(n, p, e, q);
  return vidx(n, p, q, e);
}

// Face-node map of the mesh format's orientation code.
static inline void flip_map(int flip, int N, int p, int q, int& p2, int& q2) {
  int a = (flip & 1) ? q : p;
  int bq = (flip & 1) ? p : q;
  p2 = (flip & 2) ? N - a : a;
  q2 = (flip & 4) ? N - bq : bq;
}

// Derivative along reference direction d of a nodal field u[P] at node (i,j,k).
static inline double dxi(const Ctx& c, const double* u, int d, int i, int j, int k) {
  int n = c.n;
  double s = 0.0;
  for (int m = 0; m < n; ++m) {
    int id = (d == 0) ? vidx(n, m, j, k) : (d == 1) ? vidx(n, i, m, k) : vidx(n, i, j, m);
    int row = (d == 0) ? i : (d == 1) ? j : k;
    s += c.b.D[row * n + m] * u[id];
  }
  return s;
}

// Geometry: node positions by interpolation of the equispaced samples, the
// Jacobian determinant from the derivative of the interpolant, and the
// contravariant metric terms in Kopriva's conservative curl form
//   (J a^d)_nc = -e_d . curl_xi( X_l grad_xi X_m ),  (nc, m, l) cyclic,
// which makes the discrete metric identities hold exactly (Sec. 3.1 mapping
// chi and its Jacobian; free-stream preservation).
static bool build_geometry(Ctx& c, int ngeo, const double* xgeo) {
  int n = c.n, P = c.P, m = ngeo + 1, mP = m * m * m;
  std::vector<double> V = equi_to_lgl(ngeo, c.b);
  c.X.assign((size_t)c.E * 3 * P, 0.0);
  c.Ja.assign((size_t)c.E * 9 * P, 0.0);
  c.J.assign((size_t)c.E * P, 0.0);
  std::vector<double> dX(9 * P), v(3 * P);
  for (int e = 0; e < c.E; ++e) {
    // Interpolation, metric terms and Jacobian are invariant under a
    // translation of the coordinates (the interpolant reproduces constants;
    // tensor-product derivatives along different directions commute), so they
    // are computed from coordinates relative to the element's first sample
    // (its corner, which is also the first LGL node); this removes the
    // cancellation that large absolute coordinates would cause.
    std::vector<double> Xrel(3 * P);
    for (int cc = 0; cc < 3; ++cc) {
      const double* g = xgeo + ((size_t)e * 3 + cc) * mP;
      const double g0 = g[0];
      double* Xo = &c.X[((size_t)e * 3 + cc) * P];
      for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
          for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int c3 = 0; c3 < m; ++c3)
              for (int b3 = 0; b3 < m; ++b3)
                for (int a3 = 0; a3 < m; ++a3)
                  s += V[i * m + a3] * V[j * m + b3] * V[k * m + c3] * (g[a3 + m * (b3 + m * c3)] - g0);
            Xrel[cc * P + vidx(n, i, j, k)] = s;
            Xo[vidx(n, i, j, k)] = s + g0;
          }
    }
    const double* Xe = Xrel.data();
    // dX[cc][d] = d X_cc / d xi_d
    for (int cc = 0; cc < 3; ++cc)
      for (int d = 0; d < 3; ++d)
        for (int k = 0; k < n; ++k)
          for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i)
              dX[(cc * 3 + d) * P + vidx(n, i, j, k)] = dxi(c, Xe + cc * P, d, i, j, k);
    for (int id = 0; id < P; ++id) {
      double a[3][3];
      for (int cc = 0; cc < 3; ++cc)
        for (int d = 0; d < 3; ++d) a[cc][d] = dX[(cc * 3 + d) * P + id];
      double det = a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1])
                 - a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0])
                 + a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
      c.J[(size_t)e * P + id] = det;
      if (!(det > 0.0)) { c.err = "non-positive Jacobian"; return false; }
    }
    for (int nc = 0; nc < 3; ++nc) {
      int mm = (nc + 1) % 3, ll = (nc + 2) % 3;
      // v_r = X_l * d X_m / d xi_r
      for (int r = 0; r < 3; ++r)
        for (int id = 0; id < P; ++id)
          v[r * P + id] = Xe[ll * P + id] * dX[(mm * 3 + r) * P + id];
      for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
          for (int i = 0; i < n; ++i) {
            int id = vidx(n, i, j, k);
            double c0 = dxi(c, &v[2 * P], 1, i, j, k) - dxi(c, &v[1 * P], 2, i, j, k);
            double c1 = dxi(c, &v[0 * P], 2, i, j, k) - dxi(c, &v[2 * P], 0, i, j, k);
            double c2 = dxi(c, &v[1 * P], 0, i, j, k) - dxi(c, &v[0 * P], 1, i, j, k);
            c.Ja[(((size_t)e * 3 + 0) * 3 + nc) * P + id] = -c0;
            c.Ja[(((size_t)e * 3 + 1) * 3 + nc) * P + id] = -c1;
            c.Ja[(((size_t)e * 3 + 2) * 3 + nc) * P + id] = -c2;
          }
    }
  }
  return true;
}

// Mortar interpolation: the Lagrange basis l_j of the node set x at the nodes
// of each half of [-1, 1], mI[h][a][j] = l_j((x_a + 2h - 1)/2).
static void mortar_table(Ctx& c, const std::vector<double>& x) {
  const int n = c.n;
  c.mI.assign((size_t)2 * n * n, 0.0);
  for (int k = 0; k < 2; ++k)
    for (int a = 0; a < n; ++a)
      for (int j = 0; j < n; ++j) {
        const double xs = 0.5 * (x[a] + 2.0 * k - 1.0);
        double l = 1.0;
        for (int m = 0; m < n; ++m)
          if (m != j) l *= (xs - x[m]) / (x[j] - x[m]);
        c.mI[((size_t)k * n + a) * n + j] = l;
      }
}

static bool build_faces(Ctx& c, const int* face_nbr) {
  int E = c.E, n = c.n, nn = n * n;
  c.nbr.assign(face_nbr, face_nbr + (size_t)E * 18);
  c.face_id.assign(E * 6, -1);
  c.master.assign(E * 6, 0);
  for (int m = 0; m < c.M; ++m) {   // every side of a mortar names it back
    const int* r = &c.mortars[(size_t)m * 14];
    bool ok = r[0] >= 0 && r[0] < E && r[1] >= 0 && r[1] < 6 &&
              c.nbr[(r[0] * 6 + r[1]) * 3] == -1 - m && c.nbr[(r[0] * 6 + r[1]) * 3 + 1] == 0;
    for (int k = 0; k < 4 && ok; ++k) {
      const int es = r[2 + 3 * k], fs = r[3 + 3 * k], fl = r[4 + 3 * k];
      ok = es >= 0 && es < E && fs >= 0 && fs < 6 && fl >= 0 && fl < 8 && c.nbr[(es * 6 + fs) * 3] == -1 - m &&
           c.nbr[(es * 6 + fs) * 3 + 1] == k;
    }
    if (!ok) { c.err = "mortar table does not match the connectivity"; return false; }
  }
  for (int e = 0; e < E; ++e)
    for (int f = 0; f < 6; ++f) {
      int e2 = c.nbr[(e * 6 + f) * 3 + 0], f2 = c.nbr[(e * 6 + f) * 3 + 1];
      int fl = c.nbr[(e * 6 + f) * 3 + 2];
      if (e2 < 0) {   // a side of mortar -1 - e2
        const int m = -1 - e2;
        if (m >= c.M || f2 < 0 || f2 > 3) { c.err = "connectivity out of range"; return false; }
        const int* r = &c.mortars[(size_t)m * 14];
        const bool big = r[0] == e && r[1] == f, small = r[2 + 3 * f2] == e && r[3 + 3 * f2] == f;
        if (!big && !small) { c.err = "connectivity not reciprocal"; return false; }
        continue;
      }
      if (e2 >= E || f2 < 0 || f2 > 5 || fl < 0 || fl > 7) { c.err = "connectivity out of range"; return false; }
      if (c.nbr[(e2 * 6 + f2) * 3 + 0] != e || c.nbr[(e2 * 6 + f2) * 3 + 1] != f) { c.err = "connectivity not reciprocal"; return false; }
    }
  int nf = 0;
  for (int e = 0; e < E; ++e)
    for (int f = 0; f < 6; ++f) {
      int e2 = c.nbr[(e * 6 + f) * 3 + 0], f2 = c.nbr[(e * 6 + f) * 3 + 1];
      // the two sides of a conforming face share one; each side of a mortar has its own
      if (e2 < 0 || e * 6 + f < e2 * 6 + f2) { c.master[e * 6 + f] = 1; c.face_id[e * 6 + f] = nf++; }
    }
  for (int e = 0; e < E; ++e)
    for (int f = 0; f < 6; ++f)
      if (!c.master[e * 6 + f]) {
        int e2 = c.nbr[(e * 6 + f) * 3 + 0], f2 = c.nbr[(e * 6 + f) * 3 + 1];
        c.face_id[e * 6 + f] = c.face_id[e2 * 6 + f2];
      }
  mortar_table(c, c.b.x);   // LGL; a Gauss-node context replaces it
  c.nfaces = nf;
  c.fn.assign((size_t)nf * 3 * nn, 0.0);
  c.fsJ.assign((size_t)nf * nn, 0.0);
  // Face geometry of the master side: n sJ = (2s-1) J a^d at the face node.
  for (int e = 0; e < E; ++e)
    for (int f = 0; f < 6; ++f) {
      if (!c.master[e * 6 + f]) continue;
      int d = f / 2, s = f % 2, id = c.face_id[e * 6 + f];
      for (int q = 0; q < n; ++q)
        for (int p = 0; p < n; ++p) {
          int node = face_vol(n, f, p, q);
          double nv[3], s2 = 0.0;
          for (int l = 0; l < 3; ++l) {
            nv[l] = (2.0 * s - 1.0) * c.Ja[(((size_t)e * 3 + d) * 3 + l) * c.P + node];
            s2 += nv[l] * nv[l];
          }
          double sJ = std::sqrt(s2);
          for (int l = 0; l < 3; ++l) c.fn[((size_t)id * 3 + l) * nn + p + n * q] = nv[l] / sJ;
          c.fsJ[(size_t)id * nn + p + n * q] = sJ;
        }
    }
  return true;
}

// ---------------------------------------------------------------------------
// Physics (Sec. 3.1, Eq. 1).
template <class T> struct Prim { T rho, u[3], p, T_; };

template <class T>
static inline Prim<T> cons2prim(const Params& pr, const T q[5]) {
  Prim<T> w;
  w.rho = q[0];
  for (int a = 0; a < 3; ++a) w.u[a] = q[1 + a] / q[0];
  T ke = 0.5 * (q[1] * w.u[0] + q[2] * w.u[1] + q[3] * w.u[2]);
  w.p = (pr.gamma - 1.0) * (q[4] - ke);
  w.T_ = w.p / (q[0] * pr.R);
  return w;
}

template <class T>
static inline void prim2cons(const Params& pr, const Prim<T>& w, T q[5]) {
  q[0] = w.rho;
  for (int a = 0; a < 3; ++a) q[1 + a] = w.rho * w.u[a];
  q[4] = w.p / (pr.gamma - 1.0) + 0.5 * w.rho * (w.u[0] * w.u[0] + w.u[1] * w.u[1] + w.u[2] * w.u[2]);
}

// Inviscid flux in the direction of the (not necessarily unit) vector nv.
template <class T>
static inline void euler_flux(const T q[5], const Prim<T>& w, const T nv[3], T out[5]) {
  T un = w.u[0] * nv[0] + w.u[1] * nv[1] + w.u[2] * nv[2];
  out[0] = q[0] * un;
  for (int a = 0; a < 3; ++a) out[1 + a] = q[1 + a] * un + w.p * nv[a];
  out[4] = (q[4] + w.p) * un;
}

// Dynamic viscosity at temperature Tt: mu0 itself, or Sutherland's (1893) law
// mu0 (Tt/T_ref)^(3/2) (T_ref + S) / (Tt + S).
template <class T>
static inline T visc_mu(const Params& pr, const T& mu0, const T& Tt) {
  if (pr.visc_law != 1) return mu0;
  T x = Tt / pr.T_ref;
  return mu0 * x * sqrt(x) * ((pr.T_ref + pr.S_suth) / (Tt + pr.S_suth));
}

// Viscous flux (stress + Fourier heat flux) in direction nv, from the lifted
// gradients g[phi*3 + l] = d phi / d x_l, phi in (u, v, w, T); mu0 is the
// reference viscosity, taken at the node's temperature by visc_mu.
template <class T>
static inline void visc_flux(const Params& pr, const Prim<T>& w, const T* g, const T& mu0,
                             const T nv[3], T out[5]) {
  const T mu = visc_mu(pr, mu0, w.T_);
  T div = g[0 * 3 + 0] + g[1 * 3 + 1] + g[2 * 3 + 2];
  T tau[3][3];
  for (int a = 0; a < 3; ++a)
    for (int bb = 0; bb < 3; ++bb) {
      tau[a][bb] = mu * (g[a * 3 + bb] + g[bb * 3 + a]);
      if (a == bb) tau[a][bb] = tau[a][bb] - (2.0 / 3.0) * mu * div;
    }
  double cp = pr.gamma * pr.R / (pr.gamma - 1.0);
  T lam = mu * (cp / pr.Pr);
  out[0] = T(0.0);
  for (int bb = 0; bb < 3; ++bb) {
    T s = T(0.0);
    for (int l = 0; l < 3; ++l) s += nv[l] * tau[l][bb];
    out[1 + bb] = s;
  }
  T e = T(0.0);
  for (int l = 0; l < 3; ++l) {
    T tu = tau[l][0] * w.u[0] + tau[l][1] * w.u[1] + tau[l][2] * w.u[2];
    e += nv[l] * (tu + lam * g[3 * 3 + l]);
  }
  out[4] = e;
}

// Logarithmic mean (a - b) / (ln a - ln b), Ismail & Roe (2009): with
// zeta = a/b, f = (zeta - 1)/(zeta + 1), u = f^2, the mean is (a + b)/(2 F)
// where F = ln(zeta)/(2 f) = 1 + u/3 + u^2/5 + u^3/7 + ...
template <class T>
static inline T log_mean(T a, T b) {
  T zeta = a / b;
  T f = (zeta - 1.0) / (zeta + 1.0);
  T u = f * f;
  T F;
  if (val(u) < 1e-4) F = 1.0 + u / 3.0 + u * u / 5.0 + u * u * u / 7.0;
  else F = log(zeta) / (2.0 * f);
  return (a + b) / (2.0 * F);
}

// Entropy-conserving, kinetic-energy-preserving two-point flux of
// Chandrashekar (2013) in direction nv (Sec. 3.1, entropy-stable DGSEM).
template <class T>
static inline void ec_flux(const Params& pr, const Prim<T>& L, const Prim<T>& Rr,
                           const T nv[3], T out[5]) {
  T bL = L.rho / (2.0 * L.p), bR = Rr.rho / (2.0 * Rr.p);
  T rho_ln = log_mean(L.rho, Rr.rho);
  T beta_ln = log_mean(bL, bR);
  T rho_av = 0.5 * (L.rho + Rr.rho);
  T beta_av = 0.5 * (bL + bR);
  T u_av[3];
  for (int a = 0; a < 3; ++a) u_av[a] = 0.5 * (L.u[a] + Rr.u[a]);
  T p_hat = rho_av / (2.0 * beta_av);
  T u2L = L.u[0] * L.u[0] + L.u[1] * L.u[1] + L.u[2] * L.u[2];
  T u2R = Rr.u[0] * Rr.u[0] + Rr.u[1] * Rr.u[1] + Rr.u[2] * Rr.u[2];
  T u2_av = 0.5 * (u2L + u2R);
  T un = u_av[0] * nv[0] + u_av[1] * nv[1] + u_av[2] * nv[2];
  T f_rho = rho_ln * un;
  out[0] = f_rho;
  for (int a = 0; a < 3; ++a) out[1 + a] = f_rho * u_av[a] + p_hat * nv[a];
  out[4] = f_rho * (1.0 / (2.0 * (pr.gamma - 1.0) * beta_ln) - 0.5 * u2_av)
         + u_av[0] * out[1] + u_av[1] * out[2] + u_av[2] * out[3];
}

// Local Lax-Friedrichs flux in unit direction nv.
template <class T>
static inline void llf_flux(const Params& pr, const T qL[5], const Prim<T>& L,
                            const T qR[5], const Prim<T>& Rr, const T nv[3], T out[5]) {
  T fL[5], fR[5];
  euler_flux(qL, L, nv, fL);
  euler_flux(qR, Rr, nv, fR);
  T cL = sqrt(pr.gamma * L.p / L.rho), cR = sqrt(pr.gamma * Rr.p / Rr.rho);
  T unL = L.u[0] * nv[0] + L.u[1] * nv[1] + L.u[2] * nv[2];
  T unR = Rr.u[0] * nv[0] + Rr.u[1] * nv[1] + Rr.u[2] * nv[2];
  T lmax = vmax_kink(abs_kink(unL, val(cL)) + cL, abs_kink(unR, val(cR)) + cR);
  for (int v = 0; v < 5; ++v) out[v] = 0.5 * (fL[v] + fR[v]) - 0.5 * lmax * (qR[v] - qL[v]);
}

// Roe's approximate Riemann solver with the entropy fix of Harten & Hyman
// (1983) in unit direction nv (the surface flux named in Sec. 3.1):
//   F = 1/2 (f(qL) + f(qR)) . n - 1/2 sum_k |lambda_k| alpha_k r_k
// with Roe averages (sqrt(rho) weights) of u and H, c^2 = (gamma-1)(H - |u|^2/2);
// acoustic speeds lambda = u_n -+ c, entropy and shear waves at u_n.  On the
// acoustic waves |lambda| is replaced by delta = max(0, lambda - lambda(qL),
// lambda(qR) - lambda) when |lambda| < delta.
template <class T>
static inline void roe_flux(const Params& pr, const T qL[5], const Prim<T>& L, const T qR[5], const Prim<T>& Rr,
                            const T nv[3], T out[5]) {
  T fL[5], fR[5];
  euler_flux(qL, L, nv, fL);
  euler_flux(qR, Rr, nv, fR);
  T sL = sqrt(L.rho), sR = sqrt(Rr.rho);
  T wl = sL / (sL + sR), wr = sR / (sL + sR);
  T HL = (qL[4] + L.p) / L.rho, HR = (qR[4] + Rr.p) / Rr.rho;
  T u[3];
  for (int a = 0; a < 3; ++a) u[a] = wl * L.u[a] + wr * Rr.u[a];
  T H = wl * HL + wr * HR;
  T q2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  T c = sqrt((pr.gamma - 1.0) * (H - 0.5 * q2));
  T rho = sL * sR;
  T un = u[0] * nv[0] + u[1] * nv[1] + u[2] * nv[2];
  T dr = Rr.rho - L.rho, dp = Rr.p - L.p;
  T du[3];
  for (int a = 0; a < 3; ++a) du[a] = Rr.u[a] - L.u[a];
  T dun = du[0] * nv[0] + du[1] * nv[1] + du[2] * nv[2];
  T a1 = (dp - rho * c * dun) / (2.0 * c * c);
  T a2 = dr - dp / (c * c);
  T a5 = (dp + rho * c * dun) / (2.0 * c * c);
  T l1 = fabs(un - c), l2 = fabs(un), l5 = fabs(un + c);
  // Harten-Hyman entropy fix on the acoustic waves
  T unL = L.u[0] * nv[0] + L.u[1] * nv[1] + L.u[2] * nv[2];
  T unR = Rr.u[0] * nv[0] + Rr.u[1] * nv[1] + Rr.u[2] * nv[2];
  T cL = sqrt(pr.gamma * L.p / L.rho), cR = sqrt(pr.gamma * Rr.p / Rr.rho);
  T d1 = vmax(vmax(T(0.0), (un - c) - (unL - cL)), (unR - cR) - (un - c));
  T d5 = vmax(vmax(T(0.0), (un + c) - (unL + cL)), (unR + cR) - (un + c));
  if (val(l1) < val(d1)) l1 = d1;
  if (val(l5) < val(d5)) l5 = d5;
  T D[5];
  // acoustic waves
  D[0] = l1 * a1 + l2 * a2 + l5 * a5;
  for (int a = 0; a < 3; ++a)
    D[1 + a] = l1 * a1 * (u[a] - c * nv[a]) + l2 * (a2 * u[a] + rho * (du[a] - dun * nv[a])) +
               l5 * a5 * (u[a] + c * nv[a]);
  T udu = u[0] * du[0] + u[1] * du[1] + u[2] * du[2];
  D[4] = l1 * a1 * (H - un * c) + l2 * (a2 * 0.5 * q2 + rho * (udu - un * dun)) + l5 * a5 * (H + un * c);
  for (int v = 0; v < 5; ++v) out[v] = 0.5 * (fL[v] + fR[v]) - 0.5 * D[v];
}

// Density-wave manufactured solution rho = 2 + A sin(pi (x+y+z-t)), u = (1,1,1),
// p = 1; its residual q_t + div F(q) worked out by hand:
//   r' = pi A cos(phi);  mass, momenta: 2 r';  energy: 3 r' - lambda Lap(T),
//   Lap(T) = 3 [pi^2 A sin(phi) / (R rho^2) + 2 r'^2 / (R rho^3)],  T = 1/(R rho).
static void mms_source(const Params& pr, const double x[3], double t, double out[5]) {
  double A = pr.mms_amp;
  double phi = M_PI * (x[0] + x[1] + x[2] - t);
  double rho = 2.0 + A * std::sin(phi);
  double rp = M_PI * A * std::cos(phi);
  double cp = pr.gamma * pr.R / (pr.gamma - 1.0);
  double lam = pr.mu * cp / pr.Pr;
  double lapT = 3.0 * (M_PI * M_PI * A * std::sin(phi) / (pr.R * rho * rho) + 2.0 * rp * rp / (pr.R * rho * rho * rho));
  out[0] = 2.0 * rp; out[1] = 2.0 * rp; out[2] = 2.0 * rp; out[3] = 2.0 * rp;
  out[4] = 3.0 * rp - lam * lapT;
}

// BR1 lifting (Sec. 3.1, Eq. 3) in strong form for the primitive scalars
// phi = (u, v, w, T) of every element:
//   g_l = (1/J) [ sum_d Ja^d_l (D_d phi) + sum_faces (phi* - phi) (n_l sJ) / w_end ],
// phi* = 1/2 (phi + phi_neighbour), n sJ the element's own outward normal.
// ---------------------------------------------------------------------------
// Mortars (Sec. 3.2.2, Algorithm 1; Kopriva 1996): a big face split into four
// quadrants k = a + 2 b that are faces of four small elements.  Values of the
// big face are interpolated to the nodes of each quadrant (numbered (pp, qq)
// in the big face's directions),
//   v_k(pp, qq) = sum_ij I_a[pp][i] I_b[qq][j] v(i, j),  I_h[x][j] = l_j((x_x + 2h - 1)/2),
// and quadrant data go back onto the big face by the projection with the
// quadrature of the node set (exact for the constant mode, so face integrals
// are kept; on Gauss nodes, exact to degree 2N+1, it is the L2 projection):
//   v(i, j) = scale / (w_i w_j) sum_k sum_{pp,qq} w_pp w_qq I_a[pp][i] I_b[qq][j] v_k(pp, qq),
// scale = 1/4 for point values (the lifting's face average), 1 for fluxes
// times sJ (a quadrant's surface element is a quarter of the big face's).
template <class T>
static void mortar_interp(const Ctx& c, const T* big, int k, T* out) {
  const int n = c.n, a = k & 1, b = k >> 1;
  const double* Ia = &c.mI[(size_t)a * n * n];
  const double* Ib = &c.mI[(size_t)b * n * n];
  for (int qq = 0; qq < n; ++qq)
    for (int pp = 0; pp < n; ++pp) {
      T s = T(0.0);
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) s += (Ia[pp * n + i] * Ib[qq * n + j]) * big[i + n * j];
      out[pp + n * qq] = s;
    }
}

template <class T>
static void mortar_project(const Ctx& c, const T* const quad[4], double scale, T* out) {
  const int n = c.n;
  const std::vector<double>& w = c.nodes == 1 ? c.g.w : c.b.w;   // the node set's quadrature
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      T s = T(0.0);
      for (int k = 0; k < 4; ++k) {
        const double* Ia = &c.mI[(size_t)(k & 1) * n * n];
        const double* Ib = &c.mI[(size_t)(k >> 1) * n * n];
        for (int qq = 0; qq < n; ++qq)
          for (int pp = 0; pp < n; ++pp)
            s += (w[pp] * w[qq] * Ia[pp * n + i] * Ib[qq * n + j]) * quad[k][pp + n * qq];
      }
      out[i + n * j] = s * (scale / (w[i] * w[j]));
    }
}

// Whether local face f of element e is the big side of mortar m.
static inline bool mortar_big(const Ctx& c, int m, int e, int f) {
  return c.mortars[(size_t)m * 14] == e && c.mortars[(size_t)m * 14 + 1] == f;
}

template <class T>
static void lifting(const Ctx& c, const T* phi, T* G) {
  int n = c.n, P = c.P, E = c.E, N = c.N;
  const std::vector<double>& D = c.b.D;
  double wend = c.b.w[0];
  // mortar face averages: on each quadrant (the small side's own node order)
  // and projected onto the big face
  const int nn = n * n;
  std::vector<T> star_s((size_t)c.M * 4 * 4 * nn), star_b((size_t)c.M * 4 * nn);
  for (int m = 0; m < c.M; ++m) {
    const int* r = &c.mortars[(size_t)m * 14];
    for (int ph = 0; ph < 4; ++ph) {
      std::vector<T> big(nn), q[4];
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) big[i + n * j] = phi[((size_t)r[0] * 4 + ph) * P + face_vol(n, r[1], i, j)];
      const T* qp[4];
      for (int k = 0; k < 4; ++k) {
        q[k].resize(nn);
        mortar_interp(c, big.data(), k, q[k].data());
        const int es = r[2 + 3 * k], fs = r[3 + 3 * k], fl = r[4 + 3 * k];
        for (int qq = 0; qq < n; ++qq)
          for (int pp = 0; pp < n; ++pp) {
            int p2, q2;
            flip_map(fl, N, pp, qq, p2, q2);
            const T st = 0.5 * (phi[((size_t)es * 4 + ph) * P + face_vol(n, fs, p2, q2)] + q[k][pp + n * qq]);
            star_s[(((size_t)m * 4 + k) * 4 + ph) * nn + p2 + n * q2] = st;
            q[k][pp + n * qq] = st;
          }
        qp[k] = q[k].data();
      }
      mortar_project(c, qp, 0.25, &star_b[((size_t)m * 4 + ph) * nn]);
    }
  }
#pragma omp parallel for schedule(dynamic, 4) if (kParallel<T>)
  for (int e = 0; e < E; ++e) {
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          int id = vidx(n, i, j, k);
          int ijk[3] = {i, j, k};
          for (int ph = 0; ph < 4; ++ph) {
            const T* f = &phi[((size_t)e * 4 + ph) * P];
            T dd[3];
            for (int d = 0; d < 3; ++d) {
              T s = T(0.0);
              for (int m = 0; m < n; ++m) {
                int mid = (d == 0) ? vidx(n, m, j, k) : (d == 1) ? vidx(n, i, m, k) : vidx(n, i, j, m);
                s += D[ijk[d] * n + m] * f[mid];
              }
              dd[d] = s;
            }
            for (int l = 0; l < 3; ++l) {
              T s = T(0.0);
              for (int d = 0; d < 3; ++d) s += c.Ja[(((size_t)e * 3 + d) * 3 + l) * P + id] * dd[d];
              G[((size_t)e * 12 + ph * 3 + l) * P + id] = s;
            }
          }
        }
    // surface part
    for (int f = 0; f < 6; ++f) {
      int d = f / 2, s = f % 2;
      int e2 = c.nbr[(e * 6 + f) * 3 + 0], f2 = c.nbr[(e * 6 + f) * 3 + 1], fl = c.nbr[(e * 6 + f) * 3 + 2];
      const int mo = e2 < 0 ? -1 - e2 : -1;
      const bool mbig = mo >= 0 && mortar_big(c, mo, e, f);
      for (int q = 0; q < n; ++q)
        for (int p = 0; p < n; ++p) {
          int id = face_vol(n, f, p, q);
          int p2 = 0, q2 = 0;
          if (mo < 0) flip_map(fl, N, p, q, p2, q2);
          const int id2 = mo < 0 ? face_vol(n, f2, p2, q2) : 0;
          for (int ph = 0; ph < 4; ++ph) {
            T mine = phi[((size_t)e * 4 + ph) * P + id];
            T star;
            if (mo < 0) star = 0.5 * (mine + phi[((size_t)e2 * 4 + ph) * P + id2]);
            else if (mbig) star = star_b[((size_t)mo * 4 + ph) * nn + p + n * q];
            else star = star_s[(((size_t)mo * 4 + f2) * 4 + ph) * nn + p + n * q];
            for (int l = 0; l < 3; ++l) {
              double nsJ = (2.0 * s - 1.0) * c.Ja[(((size_t)e * 3 + d) * 3 + l) * P + id];
              G[((size_t)e * 12 + ph * 3 + l) * P + id] += (star - mine) * (nsJ / wend);
            }
          }
        }
    }
    for (int r = 0; r < 12; ++r)
      for (int id = 0; id < P; ++id)
        G[((size_t)e * 12 + r) * P + id] = G[((size_t)e * 12 + r) * P + id] / c.J[(size_t)e * P + id];
  }
}

// Split-form advective volume term of element e (Sec. 3.1, entropy-stable
// DGSEM):  acc_i += sum_d sum_m 2 D_{i m} F#_d(q_i, q_m),
// F#_d evaluated with the averaged metric 1/2 (Ja^d_i + Ja^d_m).
template <class T>
static void volume_advective(const Ctx& c, int e, const Prim<T>* W, T* acc) {
  const Params& pr = c.prm;
  int n = c.n, P = c.P;
  const std::vector<double>& D = c.b.D;
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        int id = vidx(n, i, j, k);
        int ijk[3] = {i, j, k};
        for (int d = 0; d < 3; ++d)
          for (int m = 0; m < n; ++m) {
            int mid = (d == 0) ? vidx(n, m, j, k) : (d == 1) ? vidx(n, i, m, k) : vidx(n, i, j, m);
            double Dim = D[ijk[d] * n + m];
            T nv[3];
            for (int l = 0; l < 3; ++l) {
              double ji = c.Ja[(((size_t)e * 3 + d) * 3 + l) * P + id];
              double jm = c.Ja[(((size_t)e * 3 + d) * 3 + l) * P + mid];
              nv[l] = T(0.5 * (ji + jm));
            }
            T fs[5];
            if (pr.vol_flux == 0) {
              ec_flux(pr, W[id], W[mid], nv, fs);
            } else {
              T qa[5], qb[5], fa[5], fb[5];
              prim2cons(pr, W[id], qa); prim2cons(pr, W[mid], qb);
              euler_flux(qa, W[id], nv, fa); euler_flux(qb, W[mid], nv, fb);
              for (int v = 0; v < 5; ++v) fs[v] = 0.5 * (fa[v] + fb[v]);
            }
            for (int v = 0; v < 5; ++v) acc[(size_t)v * P + id] += 2.0 * Dim * fs[v];
          }
      }
}

// Viscous volume term of element e:  acc_i -= sum_d sum_m D_{i m} (f_v . Ja^d)_m.
template <class T>
static void volume_viscous(const Ctx& c, int e, const Prim<T>* W, const T* G, T mu, T* acc) {
  const Params& pr = c.prm;
  int n = c.n, P = c.P;
  const std::vector<double>& D = c.b.D;
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        int id = vidx(n, i, j, k);
        int ijk[3] = {i, j, k};
        for (int d = 0; d < 3; ++d)
          for (int m = 0; m < n; ++m) {
            int mid = (d == 0) ? vidx(n, m, j, k) : (d == 1) ? vidx(n, i, m, k) : vidx(n, i, j, m);
            double Dim = D[ijk[d] * n + m];
            T nvm[3], gm[12], fv[5];
            for (int l = 0; l < 3; ++l) nvm[l] = T(c.Ja[(((size_t)e * 3 + d) * 3 + l) * P + mid]);
            for (int r = 0; r < 12; ++r) gm[r] = G[(size_t)r * P + mid];
            visc_flux(pr, W[mid], gm, mu, nvm, fv);
            for (int v = 0; v < 5; ++v) acc[(size_t)v * P + id] -= Dim * fv[v];
          }
      }
}

// ---------------------------------------------------------------------------
// FV sub-cell shock capturing (Sec. 3.1: a 2nd-order FV operator on (N+1)^3
// sub-cells replaces the DG operator of troubled elements), FP64 only.  The
// data of one evaluation; the functions follow the Gauss section below.
struct FVData {
  int n = 0;
  double h = 0.0;                  // sub-cell width 2/n in reference space
  std::vector<double> V, Vi;       // [n][n]: J-weighted means of the nodal interpolant, its inverse
  std::vector<double> L;           // [n+1][n]: LGL Lagrange values at the sub-cell planes
  std::vector<double> Jb;          // [e][P]: sub-cell mean of J (sub-cell volume / h^3)
  std::vector<double> Ub;          // [e][5][P]: sub-cell means of U
  std::vector<double> Gb;          // [e][12][P]: sub-cell means of the lifted gradients
  std::vector<double> S;           // [e][d][plane][n*n][3]: sub-face area vectors (+xi_d)
  std::vector<double> Fb;          // [face][n*n][5]: master-outward flux of each boundary sub-face
  const double* U = nullptr;       // the nodal state and lifted gradients (DG traces of mixed faces)
  const double* G = nullptr;
  const double* Uf = nullptr;      // Gauss nodes: face values [e][6][5][n*n] and [e][6][12][n*n]
  const double* Gf = nullptr;
};
static void fv_prepare(const Ctx& c, const double* U, const double* G, FVData& fv);
static void fv_faces(const Ctx& c, FVData& fv, double* Fs);
static void fv_elements(const Ctx& c, const FVData& fv, double* Ut, double t);

// ---------------------------------------------------------------------------
// U_t = R(U): BR1 lifting, face fluxes, split-form volume integral, surface
// integral and Jacobian scaling (Sec. 3.1, Eqs. 2-3), in strong form:
//   g_l = (1/J) [ sum_d Ja^d_l d_d phi + sum_faces (phi* - phi) (n_l sJ) / w_end ]
//   V   = sum_d [ sum_m 2 D_im F#_d(q_i, q_m) - sum_m D_im (f_v . Ja^d)_m ]
//   S   = sum_faces [ F*_out - (f - f_v)(q_i, g_i) . (n sJ) ] / w_end
//   U_t = -(V + S) / J + Q
template <class T>
static void rhs(const Ctx& c, const T* U, T* Ut, double t, T mu) {
  const Params& pr = c.prm;
  int n = c.n, P = c.P, E = c.E, N = c.N, nn = n * n;
  const std::vector<double>& D = c.b.D;
  double wend = c.b.w[0];
  std::vector<Prim<T>> W((size_t)E * P);
  std::vector<T> phi((size_t)E * 4 * P);       // [e][4][P]: u, v, w, T
#pragma omp parallel for schedule(static) if (kParallel<T>)
  for (int e = 0; e < E; ++e)
    for (int id = 0; id < P; ++id) {
      T q[5];
      for (int v = 0; v < 5; ++v) q[v] = U[((size_t)e * 5 + v) * P + id];
      Prim<T> w = cons2prim(pr, q);
      W[(size_t)e * P + id] = w;
      phi[((size_t)e * 4 + 0) * P + id] = w.u[0];
      phi[((size_t)e * 4 + 1) * P + id] = w.u[1];
      phi[((size_t)e * 4 + 2) * P + id] = w.u[2];
      phi[((size_t)e * 4 + 3) * P + id] = w.T_;
    }
  // --- BR1 lifting
  std::vector<T> G((size_t)E * 12 * P);        // [e][phi*3+l][P]
  lifting(c, phi.data(), G.data());
  auto grad_at = [&](int e, int id, T g[12]) {
    for (int r = 0; r < 12; ++r) g[r] = G[((size_t)e * 12 + r) * P + id];
  };
  auto q_at = [&](int e, int id, T q[5]) {
    for (int v = 0; v < 5; ++v) q[v] = U[((size_t)e * 5 + v) * P + id];
  };
  // --- face fluxes on master faces: F* = (F_adv - F_visc) sJ, master orientation
  std::vector<T> Fs((size_t)c.nfaces * 5 * nn);
#pragma omp parallel for schedule(dynamic, 4) if (kParallel<T>)
  for (int e = 0; e < E; ++e)
    for (int f = 0; f < 6; ++f) {
      if (!c.master[e * 6 + f]) continue;
      int fid = c.face_id[e * 6 + f];
      int e2 = c.nbr[(e * 6 + f) * 3 + 0], f2 = c.nbr[(e * 6 + f) * 3 + 1], fl = c.nbr[(e * 6 + f) * 3 + 2];
      if (e2 < 0) continue;   // a mortar side: below
      for (int q = 0; q < n; ++q)
        for (int p = 0; p < n; ++p) {
          int id = face_vol(n, f, p, q);
          int p2, q2;
          flip_map(fl, N, p, q, p2, q2);
          int id2 = face_vol(n, f2, p2, q2);
          T qL[5], qR[5], gL[12], gR[12];
          q_at(e, id, qL); q_at(e2, id2, qR);
          grad_at(e, id, gL); grad_at(e2, id2, gR);
          const Prim<T>& L = W[(size_t)e * P + id];
          const Prim<T>& Rr = W[(size_t)e2 * P + id2];
          T nv[3];
          for (int l = 0; l < 3; ++l) nv[l] = T(c.fn[((size_t)fid * 3 + l) * nn + p + n * q]);
          double sJ = c.fsJ[(size_t)fid * nn + p + n * q];
          T fa[5], fvL[5], fvR[5];
          if (pr.surf_flux == 1) ec_flux(pr, L, Rr, nv, fa);
          else if (pr.surf_flux == 2) roe_flux(pr, qL, L, qR, Rr, nv, fa);
          else llf_flux(pr, qL, L, qR, Rr, nv, fa);
          visc_flux(pr, L, gL, mu, nv, fvL);
          visc_flux(pr, Rr, gR, mu, nv, fvR);
          for (int v = 0; v < 5; ++v)
            Fs[((size_t)fid * 5 + v) * nn + p + n * q] = (fa[v] - 0.5 * (fvL[v] + fvR[v])) * sJ;
        }
    }
  // --- mortars: fluxes on the quadrants (the small side's normal and surface
  // element, the big side's state and gradients interpolated), the big face's
  // flux their projection, pointing out of the big element
  for (int m = 0; m < c.M; ++m) {
    const int* r = &c.mortars[(size_t)m * 14];
    const int fidB = c.face_id[r[0] * 6 + r[1]];
    std::vector<T> big((size_t)17 * nn), qi((size_t)17 * nn), Fq((size_t)4 * 5 * nn);
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        const int id = face_vol(n, r[1], i, j);
        for (int v = 0; v < 5; ++v) big[(size_t)v * nn + i + n * j] = U[((size_t)r[0] * 5 + v) * P + id];
        for (int rr = 0; rr < 12; ++rr) big[(size_t)(5 + rr) * nn + i + n * j] = G[((size_t)r[0] * 12 + rr) * P + id];
      }
    for (int k = 0; k < 4; ++k) {
      const int es = r[2 + 3 * k], fs = r[3 + 3 * k], fl = r[4 + 3 * k];
      const int fidS = c.face_id[es * 6 + fs];
      for (int x = 0; x < 17; ++x) mortar_interp(c, &big[(size_t)x * nn], k, &qi[(size_t)x * nn]);
      for (int qq = 0; qq < n; ++qq)
        for (int pp = 0; pp < n; ++pp) {
          int p2, q2;
          flip_map(fl, N, pp, qq, p2, q2);
          const int id = face_vol(n, fs, p2, q2), o = p2 + n * q2;
          T qL[5], qR[5], gL[12], gR[12];
          q_at(es, id, qL);
          grad_at(es, id, gL);
          for (int v = 0; v < 5; ++v) qR[v] = qi[(size_t)v * nn + pp + n * qq];
          for (int rr = 0; rr < 12; ++rr) gR[rr] = qi[(size_t)(5 + rr) * nn + pp + n * qq];
          const Prim<T>& L = W[(size_t)es * P + id];
          const Prim<T> Rr = cons2prim(pr, qR);
          T nv[3];
          for (int l = 0; l < 3; ++l) nv[l] = T(c.fn[((size_t)fidS * 3 + l) * nn + o]);
          const double sJ = c.fsJ[(size_t)fidS * nn + o];
          T fa[5], fvL[5], fvR[5];
          if (pr.surf_flux == 1) ec_flux(pr, L, Rr, nv, fa);
          else if (pr.surf_flux == 2) roe_flux(pr, qL, L, qR, Rr, nv, fa);
          else llf_flux(pr, qL, L, qR, Rr, nv, fa);
          visc_flux(pr, L, gL, mu, nv, fvL);
          visc_flux(pr, Rr, gR, mu, nv, fvR);
          for (int v = 0; v < 5; ++v) {
            const T F = (fa[v] - 0.5 * (fvL[v] + fvR[v])) * sJ;
            Fs[((size_t)fidS * 5 + v) * nn + o] = F;
            Fq[((size_t)k * 5 + v) * nn + pp + n * qq] = -F;   // out of the big element
          }
        }
    }
    for (int v = 0; v < 5; ++v) {
      const T* qp[4] = {&Fq[(size_t)(0 * 5 + v) * nn], &Fq[(size_t)(1 * 5 + v) * nn], &Fq[(size_t)(2 * 5 + v) * nn],
                        &Fq[(size_t)(3 * 5 + v) * nn]};
      mortar_project(c, qp, 1.0, &Fs[((size_t)fidB * 5 + v) * nn]);
    }
  }
  // --- FV sub-cell elements: faces with an FV side take the sub-face fluxes
  // (on a DG side converted to face nodes), flagged elements the FV residual
  bool use_fv = false;
  FVData fv;
  if constexpr (std::is_same<T, double>::value) {
    use_fv = !c.fv_mask.empty();
    if (use_fv) {
      fv_prepare(c, U, G.data(), fv);
      fv_faces(c, fv, Fs.data());
    }
  }
  // --- volume integral, surface integral, Jacobian
#pragma omp parallel for schedule(dynamic, 2) if (kParallel<T>)
  for (int e = 0; e < E; ++e) {
    if (use_fv && c.fv_mask[e]) continue;
    std::vector<T> acc((size_t)5 * P, T(0.0));
    volume_advective(c, e, &W[(size_t)e * P], acc.data());
    volume_viscous(c, e, &W[(size_t)e * P], &G[(size_t)e * 12 * P], mu, acc.data());
    // surface integral
    for (int f = 0; f < 6; ++f) {
      int d = f / 2, s = f % 2;
      int fid = c.face_id[e * 6 + f];
      int ism = c.master[e * 6 + f];
      int fl = c.nbr[(e * 6 + f) * 3 + 2];
      for (int q = 0; q < n; ++q)
        for (int p = 0; p < n; ++p) {
          int id = face_vol(n, f, p, q);
          T Fout[5];
          if (ism) {
            for (int v = 0; v < 5; ++v) Fout[v] = Fs[((size_t)fid * 5 + v) * nn + p + n * q];
          } else {
            int p2, q2;
            flip_map(fl, N, p, q, p2, q2);
            for (int v = 0; v < 5; ++v) Fout[v] = -Fs[((size_t)fid * 5 + v) * nn + p2 + n * q2];
          }
          T nsJ[3];
          for (int l = 0; l < 3; ++l) nsJ[l] = T((2.0 * s - 1.0) * c.Ja[(((size_t)e * 3 + d) * 3 + l) * P + id]);
          T qi[5], gi[12], fa[5], fv[5];
          q_at(e, id, qi);
          grad_at(e, id, gi);
          euler_flux(qi, W[(size_t)e * P + id], nsJ, fa);
          visc_flux(pr, W[(size_t)e * P + id], gi, mu, nsJ, fv);
          for (int v = 0; v < 5; ++v)
            acc[(size_t)v * P + id] += (Fout[v] - (fa[v] - fv[v])) / wend;
        }
    }
    for (int id = 0; id < P; ++id) {
      double Qs[5] = {0, 0, 0, 0, 0};
      if (pr.source == 1) {
        double x[3] = {c.X[((size_t)e * 3 + 0) * P + id], c.X[((size_t)e * 3 + 1) * P + id], c.X[((size_t)e * 3 + 2) * P + id]};
        mms_source(pr, x, t, Qs);
      }
      for (int v = 0; v < 5; ++v)
        Ut[((size_t)e * 5 + v) * P + id] = -acc[(size_t)v * P + id] / c.J[(size_t)e * P + id] + Qs[v];
    }
  }
  if constexpr (std::is_same<T, double>::value) {
    if (use_fv) fv_elements(c, fv, Ut, t);
  }
}

// LSERK4-5 of Carpenter & Kennedy (1994), 2N storage (Sec. 3.1, RK4-5).
static const double RK_A[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                               -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
static const double RK_B[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                               1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                               2277821191437.0 / 14882151754819.0};
static const double RK_C[5] = {0.0, 1432997174477.0 / 9575080441755.0, 2526269341429.0 / 6820363962896.0,
                               2006345519317.0 / 3224310063776.0, 2802321613138.0 / 2924317926251.0};

// RK4-14 of Niegemann, Diehl & Busch (2012), 2N storage, fourteen stages
// (the paper's alternative scheme, Sec. 3.1), to the published sixteen digits.
static const double RK14_A[14] = {0.0, -0.7188012108672410, -0.7785331173421570, -0.0053282796654044,
                                  -0.8552979934029281, -3.9564138245774565, -1.5780575380587385,
                                  -2.0837094552574054, -0.7483334182761610, -0.7032861106563359,
                                  0.0013917096117681, -0.0932075369637460, -0.9514200470875948,
                                  -7.1151571693922548};
static const double RK14_B[14] = {0.0367762454319673, 0.3136296607553959, 0.1531848691869027, 0.0030097086818182,
                                  0.3326293790646110, 0.2440251405350864, 0.3718879239592277, 0.6204126221582444,
                                  0.1524043173028741, 0.0760894927419266, 0.0077604214040978, 0.0024647284755382,
                                  0.0780348340049386, 5.5059777270269628};
static const double RK14_C[14] = {0.0, 0.0367762454319673, 0.1249685262725025, 0.2446177702277698,
                                  0.2476149531070420, 0.2969311120382472, 0.3978149645802642,
                                  0.5270854589440328, 0.6981269994175695, 0.8190890835352128,
                                  0.8527059887098624, 0.8604711817462826, 0.8627060376969976,
                                  0.8734213127600976};

template <class T>
static void rhs_lg(const Ctx& c, const T* U, T* Ut, double t, T mu);
static void state_persson(const Ctx& c, const double* U, int var, double* out);

// Whether element e has a mortar face (a 2:1 face, Algorithm 1).  The mortar
// maps act on DG traces, so such an element stays a DG element: the FV mask
// may not flag it and the switching keeps it DG (a reading; the paper does
// not treat FV sub-cells at mortars).
static bool touches_mortar(const Ctx& c, int e) {
  for (int f = 0; f < 6; ++f)
    if (c.nbr[(e * 6 + f) * 3] < 0) return true;
  return false;
}

// Automatic switching of troubled cells (Sec. 3.1: the modal indicator marks
// the DG elements that the FV sub-cell operator takes over; Sec. 3.2.2 names
// the switch as a step of its own): before R(U) is evaluated, element e
// becomes an FV element where log10 eta_e > sw_up, a DG element where
// log10 eta_e < sw_low, and keeps its representation in between.  The state
// stays nodal in both representations, so the switch converts no data; but
// the nodal polynomial of an FV element's sub-cell means may leave the
// admissible states where its means do not, so an element goes to DG only
// with positive density and pressure at every node, and a DG element
// without them goes to FV whatever its indicator says.
static void fv_switch(const Ctx& c, const double* U) {
  std::vector<double> eta(c.E);
  state_persson(c, U, c.sw_var, eta.data());
  if (c.fv_mask.empty()) c.fv_mask.assign(c.E, 0);
  const int P = c.P;
  for (int e = 0; e < c.E; ++e) {
    bool admissible = true;
    for (int id = 0; id < P; ++id) {
      double qs[5];
      for (int v = 0; v < 5; ++v) qs[v] = U[((size_t)e * 5 + v) * P + id];
      const Prim<double> w = cons2prim(c.prm, qs);
      if (!(w.rho > 0.0 && w.p > 0.0)) admissible = false;
    }
    const double l = eta[e] > 0.0 ? std::log10(eta[e]) : -HUGE_VAL;
    if (c.M > 0 && touches_mortar(c, e)) { c.fv_mask[e] = 0; continue; }
    c.sw_margin = std::min(c.sw_margin, std::min(std::fabs(l - c.sw_up), std::fabs(l - c.sw_low)));
    if (l > c.sw_up || !admissible) c.fv_mask[e] = 1;
    else if (l < c.sw_low) c.fv_mask[e] = 0;
  }
}

// R(U) on the context's node set (the switching of troubled cells and the
// FV elements are FP64 only).
template <class T>
static void rhs_any(const Ctx& c, const T* U, T* Ut, double t, T mu) {
  if constexpr (std::is_same<T, double>::value) {
    if (c.sw_on) fv_switch(c, U);
  }
  if (c.nodes == 1) { rhs_lg(c, U, Ut, t, mu); return; }
  rhs(c, U, Ut, t, mu);
}

// nsteps steps of the context's 2N-storage scheme (RK4-5 or RK4-14).
template <class T>
static void rk_steps(const Ctx& c, T* U, double t, double dt, int nsteps, T mu) {
  size_t len = (size_t)c.E * 5 * c.P;
  const int ns = c.rk == 1 ? 14 : 5;
  const double* rA = c.rk == 1 ? RK14_A : RK_A;
  const double* rB = c.rk == 1 ? RK14_B : RK_B;
  const double* rC = c.rk == 1 ? RK14_C : RK_C;
  std::vector<T> G(len), Ut(len);
  for (int st = 0; st < nsteps; ++st) {
    for (size_t a = 0; a < len; ++a) G[a] = T(0.0);
    for (int s = 0; s < ns; ++s) {
      rhs_any(c, U, Ut.data(), t + rC[s] * dt, mu);
      for (size_t a = 0; a < len; ++a) {
        G[a] = rA[s] * G[a] + dt * Ut[a];
        U[a] = U[a] + rB[s] * G[a];
      }
    }
    t += dt;
  }
}


// ---------------------------------------------------------------------------
// Legendre-Gauss collocation: the weak form of Sec. 3.1 (Eq. 2) with the
// lifting of Eq. 3, the N+1 Gauss points per direction serving as
// interpolation and quadrature nodes.  There is no split form on these nodes:
// the volume integral takes the pointwise contravariant flux, and the face
// values are interpolated from the element (no node lies on a face).
//
// Geometry (reading): the curl-form metric terms and the node positions are
// built on the LGL nodes of degree N as for the LGL operator, then evaluated
// at the Gauss nodes and at the Gauss points of each face from that same
// polynomial.  The face values seen from both sides then agree, and the
// discrete metric identities hold for the polynomial, so a uniform state
// stays uniform.

// P_n and P_n' at an interior point x by the three-term recurrence.
static void legendre_p(int n, double x, double& Pn, double& dPn) {
  double p0 = 1.0, p1 = x;
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1; p1 = p2;
  }
  Pn = (n == 0) ? 1.0 : p1;
  dPn = (n == 0) ? 0.0 : n * (x * p1 - p0) / (x * x - 1.0);
}

static double lagrange(const std::vector<double>& xs, int j, double x) {
  double l = 1.0;
  for (size_t k = 0; k < xs.size(); ++k)
    if ((int)k != j) l *= (x - xs[k]) / (xs[j] - xs[k]);
  return l;
}

static GaussBasis make_gauss_basis(int N, const Basis& lgl) {
  GaussBasis g; g.N = N; g.n = N + 1;
  int n = N + 1;
  g.x.assign(n, 0.0); g.w.assign(n, 0.0); g.D.assign(n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double xj = -std::cos(M_PI * (j + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double Pn, dPn;
      legendre_p(n, xj, Pn, dPn);
      double dx = -Pn / dPn;
      xj += dx;
      if (std::fabs(dx) <= 1e-16 * std::max(1.0, std::fabs(xj))) break;
    }
    g.x[j] = xj;
  }
  for (int j = 0; j < n / 2; ++j) {   // exact symmetry about 0
    double m = 0.5 * (g.x[n - 1 - j] - g.x[j]);
    g.x[j] = -m; g.x[n - 1 - j] = m;
  }
  if (n % 2 == 1) g.x[n / 2] = 0.0;
  for (int j = 0; j < n; ++j) {
    double Pn, dPn;
    legendre_p(n, g.x[j], Pn, dPn);
    g.w[j] = 2.0 / ((1.0 - g.x[j] * g.x[j]) * dPn * dPn);
  }
  std::vector<double> lam(n, 1.0);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k)
      if (k != j) lam[j] /= (g.x[j] - g.x[k]);
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      double d = (lam[j] / lam[i]) / (g.x[i] - g.x[j]);
      g.D[i * n + j] = d;
      s += d;
    }
    g.D[i * n + i] = -s;
  }
  g.lm.resize(n); g.lp.resize(n);
  for (int j = 0; j < n; ++j) { g.lm[j] = lagrange(g.x, j, -1.0); g.lp[j] = lagrange(g.x, j, 1.0); }
  g.VL.resize(n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) g.VL[i * n + j] = lagrange(lgl.x, j, g.x[i]);
  return g;
}

// Volume node with index i along direction d and face-local indices (p, q)
// along the two other directions in increasing order (the face_vol convention).
static inline int line_node(int n, int d, int i, int p, int q) {
  if (d == 0) return vidx(n, i, p, q);
  if (d == 1) return vidx(n, p, i, q);
  return vidx(n, p, q, i);
}

// Replace the LGL geometry of the context by its values at the Gauss nodes
// (volume) and Gauss face points (master-side normals and surface elements).
static void gauss_geometry(Ctx& c) {
  int n = c.n, P = c.P, nn = n * n;
  const std::vector<double>& V = c.g.VL;
  auto interp3 = [&](const double* in, double* out) {   // LGL nodal -> Gauss nodal
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          double s = 0.0;
          for (int c3 = 0; c3 < n; ++c3)
            for (int b3 = 0; b3 < n; ++b3)
              for (int a3 = 0; a3 < n; ++a3)
                s += V[i * n + a3] * V[j * n + b3] * V[k * n + c3] * in[vidx(n, a3, b3, c3)];
          out[vidx(n, i, j, k)] = s;
        }
  };
  std::vector<double> X((size_t)c.E * 3 * P), Ja((size_t)c.E * 9 * P), J((size_t)c.E * P);
  std::vector<double> fn((size_t)c.nfaces * 3 * nn), fsJ((size_t)c.nfaces * nn);
  std::vector<double> rel(P), dX(9 * P), dXg(9 * P);
  for (int e = 0; e < c.E; ++e) {
    for (int cc = 0; cc < 3; ++cc) {
      const double* xl = &c.X[((size_t)e * 3 + cc) * P];
      interp3(xl, &X[((size_t)e * 3 + cc) * P]);
      // derivative of the interpolant (translation invariant: relative coordinates)
      for (int id = 0; id < P; ++id) rel[id] = xl[id] - xl[0];
      for (int d = 0; d < 3; ++d)
        for (int k = 0; k < n; ++k)
          for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) dX[(cc * 3 + d) * P + vidx(n, i, j, k)] = dxi(c, rel.data(), d, i, j, k);
    }
    for (int r = 0; r < 9; ++r) {
      interp3(&dX[(size_t)r * P], &dXg[(size_t)r * P]);
      interp3(&c.Ja[((size_t)e * 9 + r) * P], &Ja[((size_t)e * 9 + r) * P]);
    }
    for (int id = 0; id < P; ++id) {
      double a[3][3];
      for (int cc = 0; cc < 3; ++cc)
        for (int d = 0; d < 3; ++d) a[cc][d] = dXg[(cc * 3 + d) * P + id];
      J[(size_t)e * P + id] = a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1])
                            - a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0])
                            + a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
    }
    for (int f = 0; f < 6; ++f) {
      if (!c.master[e * 6 + f]) continue;
      int d = f / 2, s = f % 2, id = c.face_id[e * 6 + f];
      for (int q = 0; q < n; ++q)
        for (int p = 0; p < n; ++p) {
          double nv[3], s2 = 0.0;
          for (int l = 0; l < 3; ++l) {
            double v = 0.0;
            for (int b3 = 0; b3 < n; ++b3)
              for (int a3 = 0; a3 < n; ++a3)
                v += V[p * n + a3] * V[q * n + b3] * c.Ja[(((size_t)e * 3 + d) * 3 + l) * P + face_vol(n, f, a3, b3)];
            nv[l] = (2.0 * s - 1.0) * v;
            s2 += nv[l] * nv[l];
          }
          double sJ = std::sqrt(s2);
          for (int l = 0; l < 3; ++l) fn[((size_t)id * 3 + l) * nn + p + n * q] = nv[l] / sJ;
          fsJ[(size_t)id * nn + p + n * q] = sJ;
        }
    }
  }
  c.X.swap(X); c.Ja.swap(Ja); c.J.swap(J); c.fn.swap(fn); c.fsJ.swap(fsJ);
  for (size_t a = 0; a < c.J.size(); ++a)
    if (!(c.J[a] > 0.0)) c.err = "non-positive Jacobian at a Gauss node";
}

// Face values of nv nodal fields of every element: out[e][f][v][p + n q] =
// sum_i l_i(+-1) field(line of face point (p, q)).
template <class T>
static void prolong_to_faces(const Ctx& c, const T* field, int nv, std::vector<T>& out) {
  int n = c.n, P = c.P, nn = n * n;
  out.assign((size_t)c.E * 6 * nv * nn, T(0.0));
  for (int e = 0; e < c.E; ++e)
    for (int f = 0; f < 6; ++f) {
      int d = f / 2;
      const std::vector<double>& l = (f % 2) ? c.g.lp : c.g.lm;
      for (int v = 0; v < nv; ++v)
        for (int q = 0; q < n; ++q)
          for (int p = 0; p < n; ++p) {
            T s = T(0.0);
            for (int i = 0; i < n; ++i) s += l[i] * field[((size_t)e * nv + v) * P + line_node(n, d, i, p, q)];
            out[(((size_t)e * 6 + f) * nv + v) * nn + p + n * q] = s;
          }
    }
}

// Outward n_l sJ of element e on its local face f at its face point (p, q):
// the master's stored normal, or its negative at the mapped point.
static inline void outward_nsJ(const Ctx& c, int e, int f, int p, int q, double nsJ[3]) {
  int n = c.n, nn = n * n, fid = c.face_id[e * 6 + f];
  int pp = p, qq = q;
  double sg = 1.0;
  if (!c.master[e * 6 + f]) {
    flip_map(c.nbr[(e * 6 + f) * 3 + 2], c.N, p, q, pp, qq);
    sg = -1.0;
  }
  double sJ = c.fsJ[(size_t)fid * nn + pp + n * qq];
  for (int l = 0; l < 3; ++l) nsJ[l] = sg * c.fn[((size_t)fid * 3 + l) * nn + pp + n * qq] * sJ;
}

// BR1 lifting in the weak form of Eq. 3 for the fields phi [e][4][P] with
// face values phif [e][6][4][nn]:
//   J g_l,i = sum_faces l_{i_d}(+-1)/w_{i_d} phi* (n_l sJ) - sum_d sum_m (w_m/w_{i_d}) D_{m i_d} (phi Ja^d_l)_m,
// phi* = (phi_own + phi_nbr)/2 at each face point.
template <class T>
static void lifting_lg(const Ctx& c, const T* phi, const std::vector<T>& phif, T* G) {
  int n = c.n, P = c.P, nn = n * n, N = c.N;
  const std::vector<double>& w = c.g.w;
  const std::vector<double>& D = c.g.D;
  // mortar face averages at the face points, as on LGL nodes: on each
  // quadrant (the small side's own point order) and projected onto the big face
  std::vector<T> star_s((size_t)c.M * 4 * 4 * nn), star_b((size_t)c.M * 4 * nn);
  for (int m = 0; m < c.M; ++m) {
    const int* r = &c.mortars[(size_t)m * 14];
    for (int ph = 0; ph < 4; ++ph) {
      const T* big = &phif[(((size_t)r[0] * 6 + r[1]) * 4 + ph) * nn];
      std::vector<T> q[4];
      const T* qp[4];
      for (int k = 0; k < 4; ++k) {
        q[k].resize(nn);
        mortar_interp(c, big, k, q[k].data());
        const int es = r[2 + 3 * k], fs = r[3 + 3 * k], fl = r[4 + 3 * k];
        for (int qq = 0; qq < n; ++qq)
          for (int pp = 0; pp < n; ++pp) {
            int p2, q2;
            flip_map(fl, N, pp, qq, p2, q2);
            const T st = 0.5 * (phif[(((size_t)es * 6 + fs) * 4 + ph) * nn + p2 + n * q2] + q[k][pp + n * qq]);
            star_s[(((size_t)m * 4 + k) * 4 + ph) * nn + p2 + n * q2] = st;
            q[k][pp + n * qq] = st;
          }
        qp[k] = q[k].data();
      }
      mortar_project(c, qp, 0.25, &star_b[((size_t)m * 4 + ph) * nn]);
    }
  }
  for (int e = 0; e < c.E; ++e) {
    std::vector<T> acc((size_t)12 * P, T(0.0));
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          int id = vidx(n, i, j, k), ijk[3] = {i, j, k};
          for (int ph = 0; ph < 4; ++ph)
            for (int l = 0; l < 3; ++l) {
              T s = T(0.0);
              for (int d = 0; d < 3; ++d) {
                int r = ijk[d];
                for (int m = 0; m < n; ++m) {
                  int mid = (d == 0) ? vidx(n, m, j, k) : (d == 1) ? vidx(n, i, m, k) : vidx(n, i, j, m);
                  s += (w[m] / w[r]) * D[m * n + r] * phi[((size_t)e * 4 + ph) * P + mid] *
                       c.Ja[(((size_t)e * 3 + d) * 3 + l) * P + mid];
                }
              }
              acc[(size_t)(ph * 3 + l) * P + id] -= s;
            }
        }
    for (int f = 0; f < 6; ++f) {
      int d = f / 2;
      int e2 = c.nbr[(e * 6 + f) * 3 + 0], f2 = c.nbr[(e * 6 + f) * 3 + 1], fl = c.nbr[(e * 6 + f) * 3 + 2];
      const std::vector<double>& lend = (f % 2) ? c.g.lp : c.g.lm;
      for (int q = 0; q < n; ++q)
        for (int p = 0; p < n; ++p) {
          int p2, q2;
          flip_map(fl, N, p, q, p2, q2);
          double nsJ[3];
          outward_nsJ(c, e, f, p, q, nsJ);
          const int mo = e2 < 0 ? -1 - e2 : -1;
          const bool mbig = mo >= 0 && mortar_big(c, mo, e, f);
          for (int ph = 0; ph < 4; ++ph) {
            T star;
            if (mo < 0) {
              T mine = phif[(((size_t)e * 6 + f) * 4 + ph) * nn + p + n * q];
              T other = phif[(((size_t)e2 * 6 + f2) * 4 + ph) * nn + p2 + n * q2];
              star = 0.5 * (mine + other);
            } else if (mbig) {
              star = star_b[((size_t)mo * 4 + ph) * nn + p + n * q];
            } else {
              star = star_s[(((size_t)mo * 4 + f2) * 4 + ph) * nn + p + n * q];
            }
            for (int i = 0; i < n; ++i) {
              int id = line_node(n, d, i, p, q);
              for (int l = 0; l < 3; ++l) acc[(size_t)(ph * 3 + l) * P + id] += lend[i] / w[i] * star * nsJ[l];
            }
          }
        }
    }
    for (int r = 0; r < 12; ++r)
      for (int id = 0; id < P; ++id) G[((size_t)e * 12 + r) * P + id] = acc[(size_t)r * P + id] / c.J[(size_t)e * P + id];
  }
}

// Lifting variables (u, v, w, T) at the nodes and at the faces (from the
// face values of the conservative state).
template <class T>
static void lg_phi(const Ctx& c, const T* U, std::vector<T>& phi, std::vector<T>& Uf, std::vector<T>& phif) {
  int P = c.P, nn = c.n * c.n;
  phi.assign((size_t)c.E * 4 * P, T(0.0));
  for (int e = 0; e < c.E; ++e)
    for (int id = 0; id < P; ++id) {
      T q[5];
      for (int v = 0; v < 5; ++v) q[v] = U[((size_t)e * 5 + v) * P + id];
      Prim<T> w = cons2prim(c.prm, q);
      for (int a = 0; a < 3; ++a) phi[((size_t)e * 4 + a) * P + id] = w.u[a];
      phi[((size_t)e * 4 + 3) * P + id] = w.T_;
    }
  prolong_to_faces(c, U, 5, Uf);
  phif.assign((size_t)c.E * 6 * 4 * nn, T(0.0));
  for (int ef = 0; ef < c.E * 6; ++ef)
    for (int pq = 0; pq < nn; ++pq) {
      T q[5];
      for (int v = 0; v < 5; ++v) q[v] = Uf[((size_t)ef * 5 + v) * nn + pq];
      Prim<T> w = cons2prim(c.prm, q);
      for (int a = 0; a < 3; ++a) phif[((size_t)ef * 4 + a) * nn + pq] = w.u[a];
      phif[((size_t)ef * 4 + 3) * nn + pq] = w.T_;
    }
}

// U_t = R(U) on Gauss nodes (Sec. 3.1, Eq. 2):
//   J U_t,i = - sum_faces l_{i_d}(+-1)/w_{i_d} F*_out + sum_d sum_m (w_m/w_{i_d}) D_{m i_d} Ft^d_m + J Q,
// Ft^d = (f - f_v)(q, g) . Ja^d, F*_out = (F_adv(q-, q+; n) - {f_v} . n) sJ with
// the element's outward n, face states and gradients from prolong_to_faces.
template <class T>
static void rhs_lg(const Ctx& c, const T* U, T* Ut, double t, T mu) {
  const Params& pr = c.prm;
  int n = c.n, P = c.P, E = c.E, N = c.N, nn = n * n;
  const std::vector<double>& w = c.g.w;
  const std::vector<double>& D = c.g.D;
  std::vector<T> phi, Uf, phif, Gf;
  lg_phi(c, U, phi, Uf, phif);
  std::vector<T> G((size_t)E * 12 * P);
  lifting_lg(c, phi.data(), phif, G.data());
  prolong_to_faces(c, G.data(), 12, Gf);
  // face fluxes on master faces, master orientation
  std::vector<T> Fs((size_t)c.nfaces * 5 * nn);
  for (int e = 0; e < E; ++e)
    for (int f = 0; f < 6; ++f) {
      if (!c.master[e * 6 + f]) continue;
      int fid = c.face_id[e * 6 + f];
      int e2 = c.nbr[(e * 6 + f) * 3 + 0], f2 = c.nbr[(e * 6 + f) * 3 + 1], fl = c.nbr[(e * 6 + f) * 3 + 2];
      if (e2 < 0) continue;   // a mortar side: below
      for (int q = 0; q < n; ++q)
        for (int p = 0; p < n; ++p) {
          int p2, q2;
          flip_map(fl, N, p, q, p2, q2);
          T qL[5], qR[5], gL[12], gR[12], nv[3];
          for (int v = 0; v < 5; ++v) {
            qL[v] = Uf[(((size_t)e * 6 + f) * 5 + v) * nn + p + n * q];
            qR[v] = Uf[(((size_t)e2 * 6 + f2) * 5 + v) * nn + p2 + n * q2];
          }
          for (int r = 0; r < 12; ++r) {
            gL[r] = Gf[(((size_t)e * 6 + f) * 12 + r) * nn + p + n * q];
            gR[r] = Gf[(((size_t)e2 * 6 + f2) * 12 + r) * nn + p2 + n * q2];
          }
          for (int l = 0; l < 3; ++l) nv[l] = T(c.fn[((size_t)fid * 3 + l) * nn + p + n * q]);
          double sJ = c.fsJ[(size_t)fid * nn + p + n * q];
          Prim<T> L = cons2prim(pr, qL), Rr = cons2prim(pr, qR);
          T fa[5], fvL[5], fvR[5];
          if (pr.surf_flux == 1) ec_flux(pr, L, Rr, nv, fa);
          else if (pr.surf_flux == 2) roe_flux(pr, qL, L, qR, Rr, nv, fa);
          else llf_flux(pr, qL, L, qR, Rr, nv, fa);
          visc_flux(pr, L, gL, mu, nv, fvL);
          visc_flux(pr, Rr, gR, mu, nv, fvR);
          for (int v = 0; v < 5; ++v)
            Fs[((size_t)fid * 5 + v) * nn + p + n * q] = (fa[v] - 0.5 * (fvL[v] + fvR[v])) * sJ;
        }
    }
  // mortars, as on LGL nodes, from the face values: fluxes on the quadrants
  // (small side's normal and surface element, big side's face values of the
  // state and gradients interpolated), the big face's flux their projection
  for (int m = 0; m < c.M; ++m) {
    const int* r = &c.mortars[(size_t)m * 14];
    const int fidB = c.face_id[r[0] * 6 + r[1]];
    std::vector<T> big((size_t)17 * nn), qi((size_t)17 * nn), Fq((size_t)4 * 5 * nn);
    for (int ij = 0; ij < nn; ++ij) {
      for (int v = 0; v < 5; ++v) big[(size_t)v * nn + ij] = Uf[(((size_t)r[0] * 6 + r[1]) * 5 + v) * nn + ij];
      for (int rr = 0; rr < 12; ++rr) big[(size_t)(5 + rr) * nn + ij] = Gf[(((size_t)r[0] * 6 + r[1]) * 12 + rr) * nn + ij];
    }
    for (int k = 0; k < 4; ++k) {
      const int es = r[2 + 3 * k], fs = r[3 + 3 * k], fl = r[4 + 3 * k];
      const int fidS = c.face_id[es * 6 + fs];
      for (int x = 0; x < 17; ++x) mortar_interp(c, &big[(size_t)x * nn], k, &qi[(size_t)x * nn]);
      for (int qq = 0; qq < n; ++qq)
        for (int pp = 0; pp < n; ++pp) {
          int p2, q2;
          flip_map(fl, N, pp, qq, p2, q2);
          const int o = p2 + n * q2;
          T qL[5], qR[5], gL[12], gR[12], nv[3];
          for (int v = 0; v < 5; ++v) {
            qL[v] = Uf[(((size_t)es * 6 + fs) * 5 + v) * nn + o];
            qR[v] = qi[(size_t)v * nn + pp + n * qq];
          }
          for (int rr = 0; rr < 12; ++rr) {
            gL[rr] = Gf[(((size_t)es * 6 + fs) * 12 + rr) * nn + o];
            gR[rr] = qi[(size_t)(5 + rr) * nn + pp + n * qq];
          }
          for (int l = 0; l < 3; ++l) nv[l] = T(c.fn[((size_t)fidS * 3 + l) * nn + o]);
          const double sJ = c.fsJ[(size_t)fidS * nn + o];
          Prim<T> L = cons2prim(pr, qL), Rr = cons2prim(pr, qR);
          T fa[5], fvL[5], fvR[5];
          if (pr.surf_flux == 1) ec_flux(pr, L, Rr, nv, fa);
          else if (pr.surf_flux == 2) roe_flux(pr, qL, L, qR, Rr, nv, fa);
          else llf_flux(pr, qL, L, qR, Rr, nv, fa);
          visc_flux(pr, L, gL, mu, nv, fvL);
          visc_flux(pr, Rr, gR, mu, nv, fvR);
          for (int v = 0; v < 5; ++v) {
            const T F = (fa[v] - 0.5 * (fvL[v] + fvR[v])) * sJ;
            Fs[((size_t)fidS * 5 + v) * nn + o] = F;
            Fq[((size_t)k * 5 + v) * nn + pp + n * qq] = -F;   // out of the big element
          }
        }
    }
    for (int v = 0; v < 5; ++v) {
      const T* qp[4] = {&Fq[(size_t)(0 * 5 + v) * nn], &Fq[(size_t)(1 * 5 + v) * nn],
                             &Fq[(size_t)(2 * 5 + v) * nn], &Fq[(size_t)(3 * 5 + v) * nn]};
      mortar_project(c, qp, 1.0, &Fs[((size_t)fidB * 5 + v) * nn]);
    }
  }
  // FV sub-cell elements (as on LGL nodes; the DG side of a mixed face
  // enters with its interpolated face values)
  constexpr bool kFP64 = std::is_same<T, double>::value;   // FV elements: FP64 only
  const bool use_fv = kFP64 && !c.fv_mask.empty();
  FVData fv;
  if constexpr (kFP64) {
    if (use_fv) {
      fv_prepare(c, U, G.data(), fv);
      fv.Uf = Uf.data();
      fv.Gf = Gf.data();
      fv_faces(c, fv, Fs.data());
    }
  }
  for (int e = 0; e < E; ++e) {
    if (use_fv && c.fv_mask[e]) continue;
    // contravariant fluxes at the nodes
    std::vector<T> Ft((size_t)3 * 5 * P);
    for (int id = 0; id < P; ++id) {
      T q[5], g[12];
      for (int v = 0; v < 5; ++v) q[v] = U[((size_t)e * 5 + v) * P + id];
      for (int r = 0; r < 12; ++r) g[r] = G[((size_t)e * 12 + r) * P + id];
      Prim<T> W = cons2prim(pr, q);
      for (int d = 0; d < 3; ++d) {
        T nv[3], fa[5], fv[5];
        for (int l = 0; l < 3; ++l) nv[l] = c.Ja[(((size_t)e * 3 + d) * 3 + l) * P + id];
        euler_flux(q, W, nv, fa);
        visc_flux(pr, W, g, mu, nv, fv);
        for (int v = 0; v < 5; ++v) Ft[((size_t)d * 5 + v) * P + id] = fa[v] - fv[v];
      }
    }
    std::vector<T> acc((size_t)5 * P, T(0.0));
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          int id = vidx(n, i, j, k), ijk[3] = {i, j, k};
          for (int d = 0; d < 3; ++d) {
            int r = ijk[d];
            for (int m = 0; m < n; ++m) {
              int mid = (d == 0) ? vidx(n, m, j, k) : (d == 1) ? vidx(n, i, m, k) : vidx(n, i, j, m);
              double c_ = (w[m] / w[r]) * D[m * n + r];
              for (int v = 0; v < 5; ++v) acc[(size_t)v * P + id] -= c_ * Ft[((size_t)d * 5 + v) * P + mid];
            }
          }
        }
    for (int f = 0; f < 6; ++f) {
      int d = f / 2, fid = c.face_id[e * 6 + f];
      const std::vector<double>& lend = (f % 2) ? c.g.lp : c.g.lm;
      for (int q = 0; q < n; ++q)
        for (int p = 0; p < n; ++p) {
          T Fout[5];
          if (c.master[e * 6 + f]) {
            for (int v = 0; v < 5; ++v) Fout[v] = Fs[((size_t)fid * 5 + v) * nn + p + n * q];
          } else {
            int p2, q2;
            flip_map(c.nbr[(e * 6 + f) * 3 + 2], N, p, q, p2, q2);
            for (int v = 0; v < 5; ++v) Fout[v] = -Fs[((size_t)fid * 5 + v) * nn + p2 + n * q2];
          }
          for (int i = 0; i < n; ++i) {
            int id = line_node(n, d, i, p, q);
            for (int v = 0; v < 5; ++v) acc[(size_t)v * P + id] += lend[i] / w[i] * Fout[v];
          }
        }
    }
    for (int id = 0; id < P; ++id) {
      double Qs[5] = {0, 0, 0, 0, 0};
      if (pr.source == 1) {
        double x[3] = {c.X[((size_t)e * 3 + 0) * P + id], c.X[((size_t)e * 3 + 1) * P + id], c.X[((size_t)e * 3 + 2) * P + id]};
        mms_source(pr, x, t, Qs);
      }
      for (int v = 0; v < 5; ++v) Ut[((size_t)e * 5 + v) * P + id] = -acc[(size_t)v * P + id] / c.J[(size_t)e * P + id] + Qs[v];
    }
  }
  if constexpr (kFP64) {
    if (use_fv) fv_elements(c, fv, Ut, t);
  }
}

// Lifted gradients on either node set (test hook and diagnostics).
// ---------------------------------------------------------------------------
// FV sub-cell operator (Sec. 3.1, which fixes the scheme by citation; the
// readings taken here, on either node set):
//  F1 sub-cells: the n^3 = (N+1)^3 equal sub-cubes of the reference element,
//     width h = 2/n; sub-cells and sub-faces are indexed like nodes and face
//     nodes (the same flip codes map sub-faces across element faces).
//  F2 unknowns: J-weighted sub-cell means of the nodal interpolant,
//     ub = V3 (J u) / V3 J with V[i][j] = (1/h) int_{cell i} l_j (exact,
//     Gauss quadrature); V3 = V (x) V (x) V is invertible, so nodal values and
//     means map one to one and the element integrals agree.
//  F3 sub-face area vectors: S = int over the sub-face of J a^d, exact for the
//     metric polynomial (interpolated to the plane along d, means across):
//     each sub-cell's surface closes exactly (curl-form metrics), which keeps
//     free streams.
//  F4 reconstruction: primitive (rho, u, v, w, p) of the means, slopes along
//     each reference direction by minmod of the two one-sided differences of
//     neighbouring sub-cells (across element faces the neighbour element's
//     sub-cell), face values w +- slope/2.
//  F5 sub-face flux: local Lax-Friedrichs in the unit direction S/|S| of the
//     reconstructed states, minus the average of the two sub-cells' viscous
//     fluxes (means of the state and of the BR1-lifted gradients), times |S|.
//  F6 residual: dub/dt = -(sum of the sub-cell's outward sub-face fluxes) /
//     (Jb h^3); back to nodes by the inverse means map, J R = V3^-1 (Jb Rb),
//     plus the manufactured source at the nodes.
//  F7 element faces with an FV side are evaluated on sub-faces with the
//     master's area vectors.  An FV side enters with its reconstructed state
//     and the viscous flux of its sub-cell means; a DG side with the means of
//     its trace over each sub-face (the face nodes on LGL nodes, the values
//     interpolated to the face points on Gauss nodes), and its face flux is
//     the nodal form F* = (V (x) V)^-1 (Fb / h^2) of the sub-face fluxes,
//     whose integral over the face equals their sum.

// Gauss-Legendre rule of n points on [-1, 1].
static void gauss_rule(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int k = 0; k < n; ++k) {
    double t = std::cos(M_PI * (k + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre_p(n, t, P, dP);
      const double step = P / dP;
      t -= step;
      if (std::fabs(step) < 1e-16) break;
    }
    double P, dP;
    legendre_p(n, t, P, dP);
    x[k] = t;
    w[k] = 2.0 / ((1.0 - t * t) * dP * dP);
  }
}

// Inverse of a small dense matrix by Gauss-Jordan elimination with partial pivoting.
static std::vector<double> invert_small(int n, const std::vector<double>& A0) {
  std::vector<double> A((size_t)n * 2 * n, 0.0);
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) A[(size_t)i * 2 * n + j] = A0[(size_t)i * n + j];
    A[(size_t)i * 2 * n + n + i] = 1.0;
  }
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(A[(size_t)r * 2 * n + col]) > std::fabs(A[(size_t)piv * 2 * n + col])) piv = r;
    for (int k = 0; k < 2 * n; ++k) std::swap(A[(size_t)col * 2 * n + k], A[(size_t)piv * 2 * n + k]);
    const double dgl = A[(size_t)col * 2 * n + col];
    for (int k = 0; k < 2 * n; ++k) A[(size_t)col * 2 * n + k] /= dgl;
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const double f = A[(size_t)r * 2 * n + col];
      for (int k = 0; k < 2 * n; ++k) A[(size_t)r * 2 * n + k] -= f * A[(size_t)col * 2 * n + k];
    }
  }
  std::vector<double> B((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) B[(size_t)i * n + j] = A[(size_t)i * 2 * n + n + j];
  return B;
}

// out = (M x M x M) in on n^3 values, i fastest.
static void apply3(int n, const std::vector<double>& M, const double* in, double* out) {
  const int P = n * n * n;
  std::vector<double> t1(P), t2(P);
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int a = 0; a < n; ++a) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += M[(size_t)a * n + i] * in[vidx(n, i, j, k)];
        t1[vidx(n, a, j, k)] = s;
      }
  for (int k = 0; k < n; ++k)
    for (int b = 0; b < n; ++b)
      for (int a = 0; a < n; ++a) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += M[(size_t)b * n + j] * t1[vidx(n, a, j, k)];
        t2[vidx(n, a, b, k)] = s;
      }
  for (int c3 = 0; c3 < n; ++c3)
    for (int b = 0; b < n; ++b)
      for (int a = 0; a < n; ++a) {
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += M[(size_t)c3 * n + k] * t2[vidx(n, a, b, k)];
        out[vidx(n, a, b, c3)] = s;
      }
}

// The means matrix V, its inverse and the Lagrange values at the sub-cell planes.
static void fv_matrices(const Ctx& c, FVData& fv) {
  const std::vector<double>& xs = c.nodes == 1 ? c.g.x : c.b.x;   // the context's node set
  const int n = c.n;
  fv.n = n;
  fv.h = 2.0 / n;
  std::vector<double> gx, gw;
  gauss_rule(n, gx, gw);
  fv.V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    const double a = -1.0 + i * fv.h;
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int q = 0; q < n; ++q) s += gw[q] * lagrange(xs, j, a + 0.5 * fv.h * (1.0 + gx[q]));
      fv.V[(size_t)i * n + j] = 0.5 * s;   // (1/h) (h/2) sum_q w_q l_j
    }
  }
  fv.Vi = invert_small(n, fv.V);
  fv.L.assign((size_t)(n + 1) * n, 0.0);
  for (int pl = 0; pl <= n; ++pl)
    for (int m = 0; m < n; ++m) fv.L[(size_t)pl * n + m] = lagrange(xs, m, -1.0 + pl * fv.h);
}

static void fv_prepare(const Ctx& c, const double* U, const double* G, FVData& fv) {
  fv_matrices(c, fv);
  fv.U = U;
  fv.G = G;
  const int n = c.n, P = c.P, E = c.E, nn = n * n;
  fv.Jb.assign((size_t)E * P, 0.0);
  fv.Ub.assign((size_t)E * 5 * P, 0.0);
  fv.Gb.assign((size_t)E * 12 * P, 0.0);
  fv.S.assign((size_t)E * 3 * (n + 1) * nn * 3, 0.0);
  std::vector<double> tmp(P), out(P);
  for (int e = 0; e < E; ++e) {
    const double* J = &c.J[(size_t)e * P];
    apply3(n, fv.V, J, &fv.Jb[(size_t)e * P]);
    for (int v = 0; v < 17; ++v) {
      const double* src = v < 5 ? &U[((size_t)e * 5 + v) * P] : &G[((size_t)e * 12 + v - 5) * P];
      for (int id = 0; id < P; ++id) tmp[id] = J[id] * src[id];
      apply3(n, fv.V, tmp.data(), out.data());
      double* dst = v < 5 ? &fv.Ub[((size_t)e * 5 + v) * P] : &fv.Gb[((size_t)e * 12 + v - 5) * P];
      for (int id = 0; id < P; ++id) dst[id] = out[id] / fv.Jb[(size_t)e * P + id];
    }
    // sub-face area vectors: J a^d at the plane (along d), means across, times h^2
    for (int d = 0; d < 3; ++d)
      for (int pl = 0; pl <= n; ++pl)
        for (int l = 0; l < 3; ++l) {
          std::vector<double> T((size_t)nn);
          for (int b = 0; b < n; ++b)
            for (int a = 0; a < n; ++a) {
              double s = 0.0;
              for (int m = 0; m < n; ++m)
                s += fv.L[(size_t)pl * n + m] * c.Ja[(((size_t)e * 3 + d) * 3 + l) * P + line_node(n, d, m, a, b)];
              T[a + n * b] = s;
            }
          for (int b = 0; b < n; ++b)
            for (int a = 0; a < n; ++a) {
              double s = 0.0;
              for (int q = 0; q < n; ++q)
                for (int p = 0; p < n; ++p) s += fv.V[(size_t)a * n + p] * fv.V[(size_t)b * n + q] * T[p + n * q];
              fv.S[((((size_t)e * 3 + d) * (n + 1) + pl) * nn + a + n * b) * 3 + l] = fv.h * fv.h * s;
            }
        }
  }
}

// Primitive (rho, u, v, w, p) of element e's sub-cell at position m along d,
// transverse (a, b); m = -1 and m = n are the neighbours' sub-cells across
// the faces 2d and 2d + 1.
static void fv_prim(const Ctx& c, const FVData& fv, int e, int d, int m, int a, int b, double w[5]) {
  const int n = c.n, N = c.N, P = c.P;
  int ee = e, cell;
  if (m < 0 || m > N) {
    const int f = 2 * d + (m > N ? 1 : 0);
    const int e2 = c.nbr[(e * 6 + f) * 3 + 0], f2 = c.nbr[(e * 6 + f) * 3 + 1], fl = c.nbr[(e * 6 + f) * 3 + 2];
    int a2, b2;
    flip_map(fl, N, a, b, a2, b2);
    ee = e2;
    cell = line_node(n, f2 / 2, (f2 % 2) * N, a2, b2);
  } else {
    cell = line_node(n, d, m, a, b);
  }
  double q[5];
  for (int v = 0; v < 5; ++v) q[v] = fv.Ub[((size_t)ee * 5 + v) * P + cell];
  const Prim<double> pw = cons2prim(c.prm, q);
  w[0] = pw.rho; w[1] = pw.u[0]; w[2] = pw.u[1]; w[3] = pw.u[2]; w[4] = pw.p;
}

static inline double minmod(double x, double y) {
  if (x * y <= 0.0) return 0.0;
  return x > 0.0 ? std::min(x, y) : std::max(x, y);
}

// Reconstructed conservative state of element e's sub-cell (m along d, (a, b))
// at its face on side s (0: -xi_d, 1: +xi_d).
static void fv_face_state(const Ctx& c, const FVData& fv, int e, int d, int m, int a, int b, int s, double q[5]) {
  double wm[5], w0[5], wp[5];
  fv_prim(c, fv, e, d, m - 1, a, b, wm);
  fv_prim(c, fv, e, d, m, a, b, w0);
  fv_prim(c, fv, e, d, m + 1, a, b, wp);
  double w[5];
  for (int v = 0; v < 5; ++v) {
    const double sl = minmod(wp[v] - w0[v], w0[v] - wm[v]);
    w[v] = w0[v] + (s ? 0.5 : -0.5) * sl;
  }
  q[0] = w[0];
  for (int a3 = 0; a3 < 3; ++a3) q[1 + a3] = w[0] * w[1 + a3];
  q[4] = w[4] / (c.prm.gamma - 1.0) + 0.5 * w[0] * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]);
}

// Viscous flux . nv of element e's sub-cell `cell` from its means.
static void cell_visc(const Ctx& c, const FVData& fv, int e, int cell, const double nv[3], double out[5]) {
  const int P = c.P;
  double m[5], g[12];
  for (int v = 0; v < 5; ++v) m[v] = fv.Ub[((size_t)e * 5 + v) * P + cell];
  for (int r = 0; r < 12; ++r) g[r] = fv.Gb[((size_t)e * 12 + r) * P + cell];
  visc_flux(c.prm, cons2prim(c.prm, m), g, c.prm.mu, nv, out);
}

// DG side of a mixed face: means over its sub-face (a, b) (in its own
// face-local indices) of its face trace -- the state and the viscous flux . nv
// at the face nodes of element e's face f.
static void dg_trace_means(const Ctx& c, const FVData& fv, int e, int f, int a, int b, const double nv[3], double q[5],
                           double fvis[5]) {
  const int n = c.n, P = c.P;
  for (int v = 0; v < 5; ++v) q[v] = fvis[v] = 0.0;
  for (int qq = 0; qq < n; ++qq)
    for (int pp = 0; pp < n; ++pp) {
      const double w = fv.V[(size_t)a * n + pp] * fv.V[(size_t)b * n + qq];
      double qn[5], g[12], fn[5];
      if (fv.Uf) {   // Gauss nodes: the values interpolated to the face points
        const int nn = n * n, fp = pp + n * qq;
        for (int v = 0; v < 5; ++v) qn[v] = fv.Uf[(((size_t)e * 6 + f) * 5 + v) * nn + fp];
        for (int r = 0; r < 12; ++r) g[r] = fv.Gf[(((size_t)e * 6 + f) * 12 + r) * nn + fp];
      } else {
        const int id = face_vol(n, f, pp, qq);
        for (int v = 0; v < 5; ++v) qn[v] = fv.U[((size_t)e * 5 + v) * P + id];
        for (int r = 0; r < 12; ++r) g[r] = fv.G[((size_t)e * 12 + r) * P + id];
      }
      visc_flux(c.prm, cons2prim(c.prm, qn), g, c.prm.mu, nv, fn);
      for (int v = 0; v < 5; ++v) {
        q[v] += w * qn[v];
        fvis[v] += w * fn[v];
      }
    }
}

// Sub-face flux through area A in the unit direction nv: LLF of the two
// states minus the average of the two viscous fluxes, times A.
static void fv_flux(const Ctx& c, const double qL[5], const double qR[5], const double fvL[5], const double fvR[5],
                    const double nv[3], double A, double out[5]) {
  const Prim<double> L = cons2prim(c.prm, qL), R = cons2prim(c.prm, qR);
  double fa[5];
  llf_flux(c.prm, qL, L, qR, R, nv, fa);
  for (int v = 0; v < 5; ++v) out[v] = (fa[v] - 0.5 * (fvL[v] + fvR[v])) * A;
}

// Faces with an FV side: master-outward sub-face fluxes.  An FV side enters
// with its reconstructed state and the viscous flux of its sub-cell means, a
// DG side (mixed face) with the sub-face means of its trace; on the DG side
// the nodal form of the sub-face fluxes replaces the DG face flux.
static void fv_faces(const Ctx& c, FVData& fv, double* Fs) {
  const int n = c.n, N = c.N, nn = n * n;
  fv.Fb.assign((size_t)c.nfaces * nn * 5, 0.0);
  for (int e = 0; e < c.E; ++e)
    for (int f = 0; f < 6; ++f) {
      if (!c.master[e * 6 + f]) continue;
      const int e2 = c.nbr[(e * 6 + f) * 3 + 0], f2 = c.nbr[(e * 6 + f) * 3 + 1], fl = c.nbr[(e * 6 + f) * 3 + 2];
      if (e2 < 0) continue;   // a mortar side: DG on both sides (touches_mortar)
      const bool fvM = c.fv_mask[e] != 0, fvS = c.fv_mask[e2] != 0;
      if (!fvM && !fvS) continue;
      const int fid = c.face_id[e * 6 + f];
      const int d = f / 2, sM = f % 2, d2 = f2 / 2, sS = f2 % 2;
      for (int b = 0; b < n; ++b)
        for (int a = 0; a < n; ++a) {
          int a2, b2;
          flip_map(fl, N, a, b, a2, b2);
          const double* Sp = &fv.S[((((size_t)e * 3 + d) * (n + 1) + sM * n) * nn + a + n * b) * 3];
          const double sg = 2.0 * sM - 1.0;
          const double A = std::sqrt(Sp[0] * Sp[0] + Sp[1] * Sp[1] + Sp[2] * Sp[2]);
          const double nv[3] = {sg * Sp[0] / A, sg * Sp[1] / A, sg * Sp[2] / A};
          double qM[5], qS[5], vM[5], vS[5];
          if (fvM) {
            fv_face_state(c, fv, e, d, sM * N, a, b, sM, qM);
            cell_visc(c, fv, e, line_node(n, d, sM * N, a, b), nv, vM);
          } else {
            dg_trace_means(c, fv, e, f, a, b, nv, qM, vM);
          }
          if (fvS) {
            fv_face_state(c, fv, e2, d2, sS * N, a2, b2, sS, qS);
            cell_visc(c, fv, e2, line_node(n, d2, sS * N, a2, b2), nv, vS);
          } else {
            dg_trace_means(c, fv, e2, f2, a2, b2, nv, qS, vS);
          }
          fv_flux(c, qM, qS, vM, vS, nv, A, &fv.Fb[((size_t)fid * nn + a + n * b) * 5]);
        }
      if (fvM && fvS) continue;
      // DG side: F* at the face nodes (master orientation), (V x V)^-1 (Fb / h^2)
      for (int v = 0; v < 5; ++v)
        for (int q = 0; q < n; ++q)
          for (int p = 0; p < n; ++p) {
            double s = 0.0;
            for (int b = 0; b < n; ++b)
              for (int a = 0; a < n; ++a)
                s += fv.Vi[(size_t)p * n + a] * fv.Vi[(size_t)q * n + b] * fv.Fb[((size_t)fid * nn + a + n * b) * 5 + v];
            Fs[((size_t)fid * 5 + v) * nn + p + n * q] = s / (fv.h * fv.h);
          }
    }
}

// FV residual of the flagged elements, mapped to their nodes.
static void fv_elements(const Ctx& c, const FVData& fv, double* Ut, double t) {
  const int n = c.n, N = c.N, P = c.P, nn = n * n;
  const double h3 = fv.h * fv.h * fv.h;
  std::vector<double> JR((size_t)5 * P), out(P);
  for (int e = 0; e < c.E; ++e) {
    if (!c.fv_mask[e]) continue;
    std::fill(JR.begin(), JR.end(), 0.0);   // sum of outward sub-face fluxes per sub-cell
    for (int d = 0; d < 3; ++d)
      for (int b = 0; b < n; ++b)
        for (int a = 0; a < n; ++a)
          for (int pl = 0; pl <= n; ++pl) {
            double F[5];   // flux through plane pl in +xi_d
            if (pl > 0 && pl < n) {
              double qL[5], qR[5];
              fv_face_state(c, fv, e, d, pl - 1, a, b, 1, qL);
              fv_face_state(c, fv, e, d, pl, a, b, 0, qR);
              const double* Sv = &fv.S[((((size_t)e * 3 + d) * (n + 1) + pl) * nn + a + n * b) * 3];
              const double A = std::sqrt(Sv[0] * Sv[0] + Sv[1] * Sv[1] + Sv[2] * Sv[2]);
              const double nv[3] = {Sv[0] / A, Sv[1] / A, Sv[2] / A};
              double vL[5], vR[5];
              cell_visc(c, fv, e, line_node(n, d, pl - 1, a, b), nv, vL);
              cell_visc(c, fv, e, line_node(n, d, pl, a, b), nv, vR);
              fv_flux(c, qL, qR, vL, vR, nv, A, F);
            } else {
              const int s = pl == n ? 1 : 0, f = 2 * d + s;
              const int fid = c.face_id[e * 6 + f];
              int am = a, bm = b;
              double sgn = 1.0;   // outward flux of this element: the master's, or minus it
              if (!c.master[e * 6 + f]) {
                flip_map(c.nbr[(e * 6 + f) * 3 + 2], N, a, b, am, bm);
                sgn = -1.0;
              }
              for (int v = 0; v < 5; ++v)
                F[v] = (2.0 * s - 1.0) * sgn * fv.Fb[((size_t)fid * nn + am + n * bm) * 5 + v];
            }
            // +F leaves the sub-cell before the plane, enters the one after
            for (int v = 0; v < 5; ++v) {
              if (pl > 0) JR[(size_t)v * P + line_node(n, d, pl - 1, a, b)] += F[v];
              if (pl < n) JR[(size_t)v * P + line_node(n, d, pl, a, b)] -= F[v];
            }
          }
    for (int v = 0; v < 5; ++v) {
      // Jb Rb h^3 = -(outward fluxes): J R at the nodes = V3^-1 (Jb Rb)
      for (int id = 0; id < P; ++id) JR[(size_t)v * P + id] = -JR[(size_t)v * P + id] / h3;
      apply3(n, fv.Vi, &JR[(size_t)v * P], out.data());
      for (int id = 0; id < P; ++id) {
        double Qs[5] = {0, 0, 0, 0, 0};
        if (c.prm.source == 1) {
          const double x[3] = {c.X[((size_t)e * 3 + 0) * P + id], c.X[((size_t)e * 3 + 1) * P + id],
                               c.X[((size_t)e * 3 + 2) * P + id]};
          mms_source(c.prm, x, t, Qs);
        }
        Ut[((size_t)e * 5 + v) * P + id] = out[id] / c.J[(size_t)e * P + id] + Qs[v];
      }
    }
  }
}

static void lifted_gradients(const Ctx& c, const double* U, double* G) {
  std::vector<double> phi, Uf, phif;
  lg_phi(c, U, phi, Uf, phif);
  lifting_lg(c, phi.data(), phif, G);
}


// Volume integrals on Gauss nodes: the same quantities as orc_integrals, with
// the Gauss weights and the weak-form lifted velocity gradient.
static void integrals_lg(const Ctx& c, const double* U, double* out) {
  int n = c.n, P = c.P;
  const Params& pr = c.prm;
  std::vector<double> G((size_t)c.E * 12 * P);
  lifted_gradients(c, U, G.data());
  double tot[5] = {0, 0, 0, 0, 0}, vol = 0.0, ek = 0.0, ens = 0.0, pmin = 1e300;
  for (int e = 0; e < c.E; ++e)
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          int id = vidx(n, i, j, k);
          double wq = c.g.w[i] * c.g.w[j] * c.g.w[k] * c.J[(size_t)e * P + id];
          double q[5];
          for (int v = 0; v < 5; ++v) q[v] = U[((size_t)e * 5 + v) * P + id];
          Prim<double> w = cons2prim(pr, q);
          for (int v = 0; v < 5; ++v) tot[v] += wq * q[v];
          vol += wq;
          ek += wq * q[0] * (w.u[0] * w.u[0] + w.u[1] * w.u[1] + w.u[2] * w.u[2]);
          pmin = std::min(pmin, w.p);
          const double* g = &G[(size_t)e * 12 * P + id];
          double om0 = g[(2 * 3 + 1) * P] - g[(1 * 3 + 2) * P];
          double om1 = g[(0 * 3 + 2) * P] - g[(2 * 3 + 0) * P];
          double om2 = g[(1 * 3 + 0) * P] - g[(0 * 3 + 1) * P];
          ens += wq * visc_mu(pr, pr.mu, w.T_) * (om0 * om0 + om1 * om1 + om2 * om2);
        }
  for (int v = 0; v < 5; ++v) out[v] = tot[v];
  out[5] = 0.5 * ek / vol;
  out[6] = ens / vol;
  out[7] = pmin;
}

// ---------------------------------------------------------------------------
// Modal troubled-cell indicator of Persson & Peraire (2006), the detector that
// marks DG elements for the FV sub-cell shock capturing (Sec. 3.1).  The
// indicator quantity q of an element, given at its n = N+1 nodes per
// direction, is expanded in the orthonormal Legendre basis
//   Lt_m(xi) = sqrt((2m + 1)/2) P_m(xi),  q(x) = sum_abc qh_abc Lt_a Lt_b Lt_c,
// the unique interpolant of the nodal values (a Vandermonde solve per
// direction), and the indicator is the share of the L2 energy in the modes
// that the truncation to degree N-1 in every direction removes:
//   eta = sum_{max(a,b,c) = N} qh_abc^2 / sum_abc qh_abc^2
// (readings: the tensor-product truncation Q_{N-1}; q = rho, p or rho p).

// Orthonormal Legendre value Lt_m(x).
static double legendre_orthonormal(int m, double x) {
  double a = 1.0, b = x;
  if (m == 0) return std::sqrt(0.5);
  for (int k = 1; k < m; ++k) {
    const double c = ((2.0 * k + 1.0) * x * b - k * a) / (k + 1.0);
    a = b; b = c;
  }
  return std::sqrt((2.0 * m + 1.0) / 2.0) * b;
}

// Inverse of the Vandermonde matrix V[i][m] = Lt_m(x_i) by Gauss-Jordan
// elimination with partial pivoting: the map from nodal values to modes.
static std::vector<double> modal_transform(const std::vector<double>& x) {
  const int n = (int)x.size();
  std::vector<double> A((size_t)n * 2 * n, 0.0);   // [V | I]
  for (int i = 0; i < n; ++i) {
    for (int m = 0; m < n; ++m) A[(size_t)i * 2 * n + m] = legendre_orthonormal(m, x[i]);
    A[(size_t)i * 2 * n + n + i] = 1.0;
  }
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(A[(size_t)r * 2 * n + col]) > std::fabs(A[(size_t)piv * 2 * n + col])) piv = r;
    for (int k = 0; k < 2 * n; ++k) std::swap(A[(size_t)col * 2 * n + k], A[(size_t)piv * 2 * n + k]);
    const double d = A[(size_t)col * 2 * n + col];
    for (int k = 0; k < 2 * n; ++k) A[(size_t)col * 2 * n + k] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const double f = A[(size_t)r * 2 * n + col];
      for (int k = 0; k < 2 * n; ++k) A[(size_t)r * 2 * n + k] -= f * A[(size_t)col * 2 * n + k];
    }
  }
  std::vector<double> Vi((size_t)n * n);
  for (int m = 0; m < n; ++m)
    for (int i = 0; i < n; ++i) Vi[(size_t)m * n + i] = A[(size_t)m * 2 * n + n + i];
  return Vi;
}

// eta of one element from its nodal values q[k][j][i].
static double persson_eta(int n, const std::vector<double>& Vi, const double* q);

static void state_persson(const Ctx& c, const double* U, int var, double* out) {
  const int n = c.n, P = c.P;
  const std::vector<double>& x = c.nodes == 1 ? c.g.x : c.b.x;
  const std::vector<double> Vi = modal_transform(x);
  std::vector<double> q(P);
  for (int e = 0; e < c.E; ++e) {
    for (int id = 0; id < P; ++id) {
      double qs[5];
      for (int v = 0; v < 5; ++v) qs[v] = U[((size_t)e * 5 + v) * P + id];
      const Prim<double> w = cons2prim(c.prm, qs);
      q[id] = var == 0 ? w.rho : (var == 1 ? w.p : w.rho * w.p);
    }
    out[e] = persson_eta(n, Vi, q.data());
  }
}

static double persson_eta(int n, const std::vector<double>& Vi, const double* q) {
  const int N = n - 1;
  double top = 0.0, all = 0.0;
  for (int c = 0; c < n; ++c)
    for (int b = 0; b < n; ++b)
      for (int a = 0; a < n; ++a) {
        double qh = 0.0;
        for (int k = 0; k < n; ++k)
          for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i)
              qh += Vi[(size_t)a * n + i] * Vi[(size_t)b * n + j] * Vi[(size_t)c * n + k] * q[i + n * (j + n * k)];
        all += qh * qh;
        if (a == N || b == N || c == N) top += qh * qh;
      }
  return all > 0.0 ? top / all : 0.0;
}

}  // namespace orc

using namespace orc;

extern "C" {

// Persson indicator of nodal fields q[E][(N+1)^3] given at the nodes x (n
// values): out[e] = eta_e.
void orc_persson_field(int N, const double* x, int E, const double* q, double* out) {
  const int n = N + 1, P = n * n * n;
  std::vector<double> xs(x, x + n);
  const std::vector<double> Vi = modal_transform(xs);
  for (int e = 0; e < E; ++e) out[e] = persson_eta(n, Vi, q + (size_t)e * P);
}

// Persson indicator of the state U of an oracle context at its own nodes
// (LGL, or Gauss for a Gauss-node context); var = 0: rho, 1: p, 2: rho p.
void orc_persson(void* h, const double* U, int var, double* out) { state_persson(*(Ctx*)h, U, var, out); }

// Create an oracle context.  prm = {gamma, R, Pr, mu, mms_amp}; returns NULL
// and fills errbuf on a bad mesh.
void* orc_create(int N, int n_elems, int ngeo, const double* xgeo, const int* face_nbr, int n_mortars,
                 const int* mortars, const double* prm, int surf_flux, int source, char* errbuf, int errlen) {
  Ctx* c = new Ctx();
  c->N = N; c->n = N + 1; c->P = c->n * c->n * c->n; c->E = n_elems;
  c->prm.gamma = prm[0]; c->prm.R = prm[1]; c->prm.Pr = prm[2]; c->prm.mu = prm[3];
  c->prm.mms_amp = prm[4];
  c->prm.visc_law = (int)prm[5]; c->prm.T_ref = prm[6]; c->prm.S_suth = prm[7];
  c->nodes = (int)prm[8];
  c->rk = (int)prm[9];
  c->prm.surf_flux = surf_flux; c->prm.source = source; c->prm.vol_flux = 0;
  if (c->prm.visc_law != 0 && c->prm.visc_law != 1) {
    if (errbuf && errlen > 0) std::snprintf(errbuf, errlen, "unknown viscosity law %d", c->prm.visc_law);
    delete c;
    return nullptr;
  }
  c->b = make_basis(N);
  if (c->nodes != 0 && c->nodes != 1) c->err = "unknown node set";
  if (c->rk != 0 && c->rk != 1) c->err = "unknown Runge-Kutta scheme";
  c->M = n_mortars > 0 ? n_mortars : 0;
  if (c->M > 0) {
    c->mortars.assign(mortars, mortars + (size_t)c->M * 14);
  }
  if (!c->err.empty() || !build_geometry(*c, ngeo, xgeo) || !build_faces(*c, face_nbr)) {
    if (errbuf && errlen > 0) std::snprintf(errbuf, errlen, "%s", c->err.c_str());
    delete c;
    return nullptr;
  }
  if (c->nodes == 1) {
    c->g = make_gauss_basis(N, c->b);
    mortar_table(*c, c->g.x);
    gauss_geometry(*c);
    if (!c->err.empty()) {
      if (errbuf && errlen > 0) std::snprintf(errbuf, errlen, "%s", c->err.c_str());
      delete c;
      return nullptr;
    }
  }
  return c;
}

void orc_destroy(void* h) { delete (Ctx*)h; }

// Host threads of the FP64 operator's loops (1 unless built with OpenMP):
// sets the count if n > 0 and returns the count in effect.
int orc_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

// Test hook: select the volume two-point flux (0: Chandrashekar, 1: central).
void orc_set_vol_flux(void* h, int kind) { ((Ctx*)h)->prm.vol_flux = kind; }

// FV sub-cell elements: mask[e] != 0 switches element e to the FV sub-cell
// operator (FP64, either node set); NULL restores the pure DG operator.
// Returns 0, or -1 if the mask flags an element with a mortar face.
int orc_set_fv_mask(void* h, const int* mask) {
  Ctx* c = (Ctx*)h;
  if (!mask) { c->fv_mask.clear(); return 0; }
  for (int e = 0; e < c->E; ++e)
    if (mask[e] && c->M > 0 && touches_mortar(*c, e)) return -1;
  c->fv_mask.assign(mask, mask + c->E);
  return 0;
}

// Automatic DG/FV switching (fv_switch) with the indicator of var (0: rho,
// 1: p, 2: rho p) against log10 thresholds up >= low; var < 0 turns it off
// (the mask stays as it is); elements with a mortar face stay DG.  Returns 0,
// or -2 for bad arguments.
int orc_set_fv_switch(void* h, int var, double log10_up, double log10_low) {
  Ctx* c = (Ctx*)h;
  if (var < 0) { c->sw_on = false; return 0; }
  if (var > 2 || !(log10_up >= log10_low)) return -2;
  c->sw_on = true;
  c->sw_var = var;
  c->sw_up = log10_up;
  c->sw_low = log10_low;
  return 0;
}

// The FV mask in effect (all zero if none); returns and resets the smallest
// distance of a log10 eta from a threshold since the last call.
double orc_fv_state(void* h, int* mask) {
  Ctx* c = (Ctx*)h;
  for (int e = 0; e < c->E; ++e) mask[e] = c->fv_mask.empty() ? 0 : c->fv_mask[e];
  const double m = c->sw_margin;
  c->sw_margin = 1e300;
  return m;
}

// Lifted gradients G [E][12][P] (row phi*3 + l = d phi / d x_l).
void orc_lifting(void* h, const double* U, double* G) {
  Ctx* c = (Ctx*)h;
  if (c->nodes == 1) { lifted_gradients(*c, U, G); return; }
  int P = c->P;
  std::vector<double> phi((size_t)c->E * 4 * P);
  for (int e = 0; e < c->E; ++e)
    for (int id = 0; id < P; ++id) {
      double q[5];
      for (int v = 0; v < 5; ++v) q[v] = U[((size_t)e * 5 + v) * P + id];
      Prim<double> w = cons2prim(c->prm, q);
      for (int a = 0; a < 3; ++a) phi[((size_t)e * 4 + a) * P + id] = w.u[a];
      phi[((size_t)e * 4 + 3) * P + id] = w.T_;
    }
  lifting(*c, phi.data(), G);
}

// Advective split-form volume term only: out [E][5][P] = V (before -1/J).
void orc_volume_term(void* h, const double* U, double* out) {
  Ctx* c = (Ctx*)h;
  int P = c->P;
  std::vector<Prim<double>> W((size_t)P);
  for (int e = 0; e < c->E; ++e) {
    for (int id = 0; id < P; ++id) {
      double q[5];
      for (int v = 0; v < 5; ++v) q[v] = U[((size_t)e * 5 + v) * P + id];
      W[id] = cons2prim(c->prm, q);
    }
    std::fill(out + (size_t)e * 5 * P, out + (size_t)(e + 1) * 5 * P, 0.0);
    volume_advective(*c, e, W.data(), out + (size_t)e * 5 * P);
  }
}

int orc_nfaces(void* h) { return ((Ctx*)h)->nfaces; }

void orc_basis(int N, double* x, double* w, double* D) {
  Basis b = make_basis(N);
  std::memcpy(x, b.x.data(), sizeof(double) * b.n);
  std::memcpy(w, b.w.data(), sizeof(double) * b.n);
  std::memcpy(D, b.D.data(), sizeof(double) * b.n * b.n);
}

// Geometry outputs: X [E][3][P], Ja [E][3][3][P], J [E][P].
void orc_geometry(void* h, double* X, double* Ja, double* J) {
  Ctx* c = (Ctx*)h;
  if (X) std::memcpy(X, c->X.data(), sizeof(double) * c->X.size());
  if (Ja) std::memcpy(Ja, c->Ja.data(), sizeof(double) * c->Ja.size());
  if (J) std::memcpy(J, c->J.data(), sizeof(double) * c->J.size());
}

void orc_time_derivative(void* h, const double* U, double* Ut, double t) {
  Ctx* c = (Ctx*)h;
  rhs_any<double>(*c, U, Ut, t, c->prm.mu);
}

// Legendre-Gauss basis of degree N: nodes, weights, D, l_j(-1), l_j(+1).
void orc_gauss_basis(int N, double* x, double* w, double* D, double* lm, double* lp) {
  GaussBasis g = make_gauss_basis(N, make_basis(N));
  int n = N + 1;
  std::memcpy(x, g.x.data(), sizeof(double) * n);
  std::memcpy(w, g.w.data(), sizeof(double) * n);
  std::memcpy(D, g.D.data(), sizeof(double) * n * n);
  std::memcpy(lm, g.lm.data(), sizeof(double) * n);
  std::memcpy(lp, g.lp.data(), sizeof(double) * n);
}

int orc_nodes(void* h) { return ((Ctx*)h)->nodes; }

// Tangent-linear: Ut = R(U) and dUt = dR/dU . dU + dR/dmu . dmu.
void orc_time_derivative_tl(void* h, const double* U, const double* dU, double dmu,
                            double* Ut, double* dUt, double t) {
  Ctx* c = (Ctx*)h;
  size_t len = (size_t)c->E * 5 * c->P;
  std::vector<Dual> Ud(len), Utd(len);
  for (size_t a = 0; a < len; ++a) Ud[a] = Dual(U[a], dU ? dU[a] : 0.0);
  rhs_any<Dual>(*c, Ud.data(), Utd.data(), t, Dual(c->prm.mu, dmu));
  for (size_t a = 0; a < len; ++a) { if (Ut) Ut[a] = Utd[a].v; if (dUt) dUt[a] = Utd[a].d; }
}

// Floating-point operations of one evaluation of R(U) by the LGL operator of
// this oracle, counted with the Counted scalar: out5 = {additions and
// subtractions, multiplications, divisions, square roots, logarithms}.
void orc_count_ops(void* h, const double* U, double t, double* out5) {
  Ctx* c = (Ctx*)h;
  for (int k = 0; k < 5; ++k) out5[k] = 0.0;
  if (c->nodes != 0) return;   // counted for the LGL operator
  size_t len = (size_t)c->E * 5 * c->P;
  std::vector<Counted> Uc(len), Utc(len);
  for (size_t a = 0; a < len; ++a) Uc[a] = Counted(U[a]);
  g_ops = OpCount();
  rhs<Counted>(*c, Uc.data(), Utc.data(), t, Counted(c->prm.mu));
  out5[0] = (double)g_ops.add; out5[1] = (double)g_ops.mul; out5[2] = (double)g_ops.div;
  out5[3] = (double)g_ops.sqrt; out5[4] = (double)g_ops.log;
}

// The same count for one two-point flux evaluation (Chandrashekar) of the
// conservative states qL, qR in direction nv.
void orc_count_ec_flux_ops(const double* prm, const double* qL, const double* qR, const double* nv, double* out5) {
  Params pr{prm[0], prm[1], prm[2], prm[3], 0, 0, 0.0, 0, 0, 1.0, 0.0};
  Counted a[5], b[5], n3[3], f[5];
  for (int k = 0; k < 5; ++k) { a[k] = Counted(qL[k]); b[k] = Counted(qR[k]); }
  for (int k = 0; k < 3; ++k) n3[k] = Counted(nv[k]);
  Prim<Counted> L = cons2prim(pr, a), Rr = cons2prim(pr, b);
  g_ops = OpCount();
  ec_flux(pr, L, Rr, n3, f);
  out5[0] = (double)g_ops.add; out5[1] = (double)g_ops.mul; out5[2] = (double)g_ops.div;
  out5[3] = (double)g_ops.sqrt; out5[4] = (double)g_ops.log;
}

void orc_rk_steps(void* h, double* U, double t, double dt, int nsteps) {
  Ctx* c = (Ctx*)h;
  rk_steps<double>(*c, U, t, dt, nsteps, c->prm.mu);
}

// Tangent-linear of nsteps LSERK steps: U and dU advanced together.
void orc_rk_steps_tl(void* h, double* U, double* dU, double dmu, double t, double dt, int nsteps) {
  Ctx* c = (Ctx*)h;
  size_t len = (size_t)c->E * 5 * c->P;
  std::vector<Dual> Ud(len);
  for (size_t a = 0; a < len; ++a) Ud[a] = Dual(U[a], dU[a]);
  rk_steps<Dual>(*c, Ud.data(), t, dt, nsteps, Dual(c->prm.mu, dmu));
  for (size_t a = 0; a < len; ++a) { U[a] = Ud[a].v; dU[a] = Ud[a].d; }
}

void orc_rk_coeffs(double* A, double* B, double* C) {
  std::memcpy(A, RK_A, sizeof(RK_A)); std::memcpy(B, RK_B, sizeof(RK_B)); std::memcpy(C, RK_C, sizeof(RK_C));
}

// Coefficients of RK4-14 (14 values each).
void orc_rk14_coeffs(double* A, double* B, double* C) {
  std::memcpy(A, RK14_A, sizeof(RK14_A)); std::memcpy(B, RK14_B, sizeof(RK14_B)); std::memcpy(C, RK14_C, sizeof(RK14_C));
}

// Two-point flux, LLF flux and log mean exposed for the pin tests.
void orc_ec_flux(const double* prm, const double* qL, const double* qR, const double* nv, double* out) {
  Params pr{prm[0], prm[1], prm[2], prm[3], 0, 0, 0.0, 0, 0, 1.0, 0.0};
  Prim<double> L = cons2prim(pr, qL), Rr = cons2prim(pr, qR);
  ec_flux(pr, L, Rr, nv, out);
}
void orc_llf_flux(const double* prm, const double* qL, const double* qR, const double* nv, double* out) {
  Params pr{prm[0], prm[1], prm[2], prm[3], 0, 0, 0.0, 0, 0, 1.0, 0.0};
  Prim<double> L = cons2prim(pr, qL), Rr = cons2prim(pr, qR);
  llf_flux(pr, qL, L, qR, Rr, nv, out);
}
void orc_roe_flux(const double* prm, const double* qL, const double* qR, const double* nv, double* out) {
  Params pr{prm[0], prm[1], prm[2], prm[3], 0, 0, 0.0, 0, 0, 1.0, 0.0};
  Prim<double> L = cons2prim(pr, qL), Rr = cons2prim(pr, qR);
  roe_flux(pr, qL, L, qR, Rr, nv, out);
}
double orc_log_mean(double a, double b) { return log_mean<double>(a, b); }

// Volume integrals (Sec. 4.2 diagnostics) with the LGL quadrature:
// out = {int rho, int rho u, int rho v, int rho w, int rho E,
//        E_k = 1/(2|Omega|) int rho |u|^2, eps_S = 1/|Omega| int mu(T) |omega|^2,
//        min p}; rho0 = U0 = L = 1, mu0 = 1/Re, mu(T) by the viscosity law.
void orc_integrals(void* h, const double* U, double* out) {
  Ctx* c = (Ctx*)h;
  if (c->nodes == 1) { integrals_lg(*c, U, out); return; }
  int n = c->n, P = c->P;
  const Params& pr = c->prm;
  // gradients from the lifting: reuse rhs machinery through a local copy
  size_t len = (size_t)c->E * 5 * P;
  (void)len;
  double tot[5] = {0, 0, 0, 0, 0}, vol = 0.0, ek = 0.0, ens = 0.0, pmin = 1e300;
  // lifted gradient of the velocity (same BR1 operator as in rhs)
  std::vector<double> phi((size_t)c->E * 3 * P);
  for (int e = 0; e < c->E; ++e)
    for (int id = 0; id < P; ++id) {
      double q[5];
      for (int v = 0; v < 5; ++v) q[v] = U[((size_t)e * 5 + v) * P + id];
      for (int a = 0; a < 3; ++a) phi[((size_t)e * 3 + a) * P + id] = q[1 + a] / q[0];
    }
  for (int e = 0; e < c->E; ++e)
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          int id = vidx(n, i, j, k);
          double wq = c->b.w[i] * c->b.w[j] * c->b.w[k] * c->J[(size_t)e * P + id];
          double q[5];
          for (int v = 0; v < 5; ++v) q[v] = U[((size_t)e * 5 + v) * P + id];
          Prim<double> w = cons2prim(pr, q);
          for (int v = 0; v < 5; ++v) tot[v] += wq * q[v];
          vol += wq;
          ek += wq * q[0] * (w.u[0] * w.u[0] + w.u[1] * w.u[1] + w.u[2] * w.u[2]);
          pmin = std::min(pmin, w.p);
        }
  // vorticity from the BR1 lifted velocity gradient
  int N = c->N;
  double wend = c->b.w[0];
  for (int e = 0; e < c->E; ++e) {
    std::vector<double> g((size_t)9 * P, 0.0);   // [a*3+l]
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          int id = vidx(n, i, j, k);
          for (int a = 0; a < 3; ++a) {
            const double* f = &phi[((size_t)e * 3 + a) * P];
            double dd[3];
            for (int d = 0; d < 3; ++d) dd[d] = dxi(*c, f, d, i, j, k);
            for (int l = 0; l < 3; ++l) {
              double s = 0.0;
              for (int d = 0; d < 3; ++d) s += c->Ja[(((size_t)e * 3 + d) * 3 + l) * P + id] * dd[d];
              g[(a * 3 + l) * P + id] = s;
            }
          }
        }
    for (int f = 0; f < 6; ++f) {
      int d = f / 2, s = f % 2;
      int e2 = c->nbr[(e * 6 + f) * 3 + 0], f2 = c->nbr[(e * 6 + f) * 3 + 1], fl = c->nbr[(e * 6 + f) * 3 + 2];
      for (int q = 0; q < n; ++q)
        for (int p = 0; p < n; ++p) {
          int id = face_vol(n, f, p, q);
          int p2, q2;
          flip_map(fl, N, p, q, p2, q2);
          int id2 = face_vol(n, f2, p2, q2);
          for (int a = 0; a < 3; ++a) {
            double mine = phi[((size_t)e * 3 + a) * P + id];
            double other = phi[((size_t)e2 * 3 + a) * P + id2];
            double star = 0.5 * (mine + other);
            for (int l = 0; l < 3; ++l) {
              double nsJ = (2.0 * s - 1.0) * c->Ja[(((size_t)e * 3 + d) * 3 + l) * P + id];
              g[(a * 3 + l) * P + id] += (star - mine) * nsJ / wend;
            }
          }
        }
    }
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          int id = vidx(n, i, j, k);
          double Jv = c->J[(size_t)e * P + id];
          double wq = c->b.w[i] * c->b.w[j] * c->b.w[k] * Jv;
          double gg[9];
          for (int r = 0; r < 9; ++r) gg[r] = g[r * P + id] / Jv;
          double om0 = gg[2 * 3 + 1] - gg[1 * 3 + 2];
          double om1 = gg[0 * 3 + 2] - gg[2 * 3 + 0];
          double om2 = gg[1 * 3 + 0] - gg[0 * 3 + 1];
          double q[5];
          for (int v = 0; v < 5; ++v) q[v] = U[((size_t)e * 5 + v) * P + id];
          // Sutherland's mu(T) needs T > 0: a node with T <= 0 (only inside an FV
          // element, whose nodal polynomial of admissible sub-cell means may
          // leave the admissible states) adds nothing
          const double Tn = cons2prim(pr, q).T_;
          const double mu_n = (pr.visc_law == 1 && Tn <= 0.0) ? 0.0 : visc_mu(pr, pr.mu, Tn);
          ens += wq * mu_n * (om0 * om0 + om1 * om1 + om2 * om2);
        }
  }
  for (int v = 0; v < 5; ++v) out[v] = tot[v];
  out[5] = 0.5 * ek / vol;
  out[6] = ens / vol;
  out[7] = pmin;
}

// Node positions [E][3][P] (interpolated geometry at the LGL nodes).
void orc_node_coords(void* h, double* X) {
  Ctx* c = (Ctx*)h;
  std::memcpy(X, c->X.data(), sizeof(double) * c->X.size());
}

// Initial states at the LGL nodes.
//  kind 0: Taylor-Green vortex (Sec. 4.2, Eq. 6) with rho0 = U0 = L = R = 1,
//          p0 = prm0, T0 = p0, rho = p / (R T0).
//  kind 1: density-wave manufactured solution at time prm0.
void orc_initial_state(void* h, int kind, double prm0, double* U) {
  Ctx* c = (Ctx*)h;
  int P = c->P;
  double g = c->prm.gamma;
  for (int e = 0; e < c->E; ++e)
    for (int id = 0; id < P; ++id) {
      double x = c->X[((size_t)e * 3 + 0) * P + id];
      double y = c->X[((size_t)e * 3 + 1) * P + id];
      double z = c->X[((size_t)e * 3 + 2) * P + id];
      double rho, u[3], p;
      if (kind == 0) {
        double p0 = prm0;
        u[0] = std::sin(x) * std::cos(y) * std::cos(z);
        u[1] = -std::cos(x) * std::sin(y) * std::cos(z);
        u[2] = 0.0;
        p = p0 + (1.0 / 16.0) * (std::cos(2.0 * x) + std::cos(2.0 * y)) * (2.0 + std::cos(2.0 * z));
        rho = p / (c->prm.R * p0);
      } else {
        rho = 2.0 + c->prm.mms_amp * std::sin(M_PI * (x + y + z - prm0));
        u[0] = u[1] = u[2] = 1.0;
        p = 1.0;
      }
      U[((size_t)e * 5 + 0) * P + id] = rho;
      for (int a = 0; a < 3; ++a) U[((size_t)e * 5 + 1 + a) * P + id] = rho * u[a];
      U[((size_t)e * 5 + 4) * P + id] = p / (g - 1.0) + 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    }
}

}  // extern "C"
