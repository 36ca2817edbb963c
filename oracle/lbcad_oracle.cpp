// lbcad_oracle.cpp -- plain FP64 CPU oracle for one hybrid lattice-Boltzmann step
// of a 3D active cholesteric droplet (Carenza, Gonnella & Negro, arXiv:2011.00287).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, import or call
// this file; it is used by tests/, by __graft_entry__.smoke() (as the checker) and by
// bench.py's cpu_baseline / --impl reference legs.  It shares no code, header, table
// or constant with the CUDA library: the D3Q19 table, the stencils, the free energy,
// the stresses and the seeded initial state are written out again here.
//
// Everything is a plain loop in double precision, one stage after another, in the
// order of the paper's model (Sec. 2, Eqs. 1-5) and scheme (Sec. 3, Eqs. 6-11).  Each
// per-site stage loop carries an OpenMP parallel-for over z, which compiles away without
// -fopenmp: every site's outputs are written by that site's iteration alone (streaming
// writes each population to one destination), so the threaded build computes the same
// numbers in the same order per site.  The stages:
//   1. stencils on Q and psi                 (Sec. 3: finite differences for the order parameters)
//   2. molecular field H = -dF/dQ            (Eq. 2, Eq. 5)
//   3. chemical potential mu = dF/dphi       (Eq. 1, Eq. 5)
//   4. stress sigma = passive + active       (Eq. 3, Eq. 4)
//   5. body force F = div sigma              (Eq. 3, Eq. 10 read as the whole div sigma)
//   6. BGK collision with Guo forcing, then streaming  (Eqs. 6-8; Eq. 7 read as BGK + Guo)
//   7. Beris-Edwards update of Q (Eq. 2) and Cahn-Hilliard update of psi (Eq. 1),
//      first-order upwind advection (Sec. 3), Euler or Heun predictor-corrector.
// Readings of the parts the paper leaves open (all are parameters):
//   * lattice D3Q19 (the paper used D3Q15); whole sigma enters as a body force, f^eq has
//     no stress term (G_i = 0 in Eq. 11).
//   * psi = phi - 1 in [-1, 1] (phi0 = 2, phi_cr = 1), so the bulk term of Eq. 5 is
//     -a psi^2/2 + b psi^4/4 with a = b; chi(phi) = chi0 + chis*phi with phi = 1 + psi.
//   * H is the symmetric traceless part of -dF/dQ and multiplies Gamma_Q (Eq. 2 read as
//     dQ/dt = ... + Gamma_Q H).
//   * the elastic energy (K/2)[(div Q)^2 + (curl Q + 2 q0 Q)^2] is used in its
//     one-constant form (K/2)(dQ)^2 + 2 K q0 Q:(curl Q) + 2 K q0^2 Q:Q, which differs by a
//     null Lagrangian: identical H, it only fixes the elastic stress Pi.
//   * active stress -zeta phi_c Q with phi_c = (1 + psi)/2 (Eq. 4 restricted to the droplet).
//   * stencils: isotropic D3Q19 gradient and Laplacian (radius 1); Hessian of psi from
//     the three-point and the four-corner differences.
//   * isotropic pressure P0 = psi*mu - f, f the free-energy density of Eq. 5.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {

// Parameters of Eqs. 1-11 (plus the readings above).  Layout mirrored by oracle/oracle.py.
typedef struct {
  double tau, rho0;
  double A0, chi0, chis, K, q0, gammaQ, xi;
  double a, b, kphi, M, W, zeta;
  double R, cx, cy, cz;   // droplet radius and centre
  double S0, noise;       // initial scalar order inside the droplet and noise amplitude
  int integrator;         // 0 = Euler, 1 = Heun predictor-corrector (Sec. 3)
  int coupling;           // 0 = advect with u(t-1), 1 = advect with u(t) of this step
  int lattice;            // LB velocity set: 19 = D3Q19, 15 = D3Q15 (Sec. 3, Fig. 1)
  int lb_form;            // 0 = whole stress as a body force (Guo), 1 = Eqs. 9-11: symmetric
                          //     stress in the equilibrium, antisymmetric stress as forcing
  int stencil;            // finite differences: 0 = isotropic D3Q19 (radius 1), 1 = fourth-order
                          //     truncation along the axes (radius 2), the other reading of Sec. 3
} orc_params;

}  // extern "C"

namespace {

const int NQ = 19;
// D3Q19 velocity set: rest, six faces, twelve edges.
const int CV[NQ][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

double wgt(int i) {
  int s = CV[i][0] * CV[i][0] + CV[i][1] * CV[i][1] + CV[i][2] * CV[i][2];
  if (s == 0) return 1.0 / 3.0;
  if (s == 1) return 1.0 / 18.0;
  return 1.0 / 36.0;
}

// D3Q15 velocity set: rest, six faces, eight corners, opposite velocities adjacent.
// Weights 2/9, 1/9, 1/72 (c_s^2 = 1/3, isotropic to fourth order like D3Q19).
const int CV15[15][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 1}, {-1, -1, -1}, {1, 1, -1}, {-1, -1, 1}, {1, -1, 1}, {-1, 1, -1}, {-1, 1, 1}, {1, -1, -1}};

double wgt15(int i) {
  int s = CV15[i][0] * CV15[i][0] + CV15[i][1] * CV15[i][1] + CV15[i][2] * CV15[i][2];
  if (s == 0) return 2.0 / 9.0;
  if (s == 1) return 1.0 / 9.0;
  return 1.0 / 72.0;
}

// The LB velocity set of a run (the finite-difference stencils always use D3Q19).
struct LBSet {
  int q;
  int c[19][3];
  double w[19];
};

LBSet lb_set(int lattice) {
  LBSet L;
  L.q = (lattice == 15) ? 15 : 19;
  for (int i = 0; i < L.q; ++i) {
    for (int a = 0; a < 3; ++a) L.c[i][a] = (L.q == 15) ? CV15[i][a] : CV[i][a];
    L.w[i] = (L.q == 15) ? wgt15(i) : wgt(i);
  }
  return L;
}

struct Box {
  int nx, ny, nz;
  long n() const { return (long)nx * ny * nz; }
  long at(int x, int y, int z) const {
    x %= nx; if (x < 0) x += nx;
    y %= ny; if (y < 0) y += ny;
    z %= nz; if (z < 0) z += nz;
    return x + (long)nx * (y + (long)ny * z);
  }
};

// Everything below is templated on the scalar type R: R = double is the oracle; R = Dual
// (a value and one tangent, defined further down) carries forward-mode derivatives through
// the same arithmetic.
template <typename R>
using M3 = R[3][3];

// Parameters promoted to R (so that zeta and q0 can carry tangents).
template <typename R>
struct PR {
  R tau, rho0, A0, chi0, chis, K, q0, gammaQ, xi, a, b, kphi, M, W, zeta;
  int integrator, coupling, lattice, lb_form, stencil;
};

template <typename R>
PR<R> promote(const orc_params& p) {
  PR<R> r;
  r.tau = p.tau; r.rho0 = p.rho0; r.A0 = p.A0; r.chi0 = p.chi0; r.chis = p.chis; r.K = p.K; r.q0 = p.q0;
  r.gammaQ = p.gammaQ; r.xi = p.xi; r.a = p.a; r.b = p.b; r.kphi = p.kphi; r.M = p.M; r.W = p.W; r.zeta = p.zeta;
  r.integrator = p.integrator;
  r.coupling = p.coupling;
  r.lattice = p.lattice;
  r.lb_form = p.lb_form;
  r.stencil = p.stencil;
  return r;
}

inline double max0(double v) { return std::fmax(v, 0.0); }
inline double min0(double v) { return std::fmin(v, 0.0); }

// Forward-mode dual number: a value and one directional derivative.  Every operation of
// the step is +, -, *, / or a comparison, so these rules differentiate it exactly; at the
// switching points of max(u, 0) and of the upwind face choice the derivative of the
// branch taken is used.
struct Dual {
  double v, d;
  Dual() : v(0.0), d(0.0) {}
  Dual(double x) : v(x), d(0.0) {}
  Dual(double x, double dx) : v(x), d(dx) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) { return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
inline Dual& operator+=(Dual& a, Dual b) { return a = a + b; }
inline Dual& operator-=(Dual& a, Dual b) { return a = a - b; }
inline Dual& operator*=(Dual& a, Dual b) { return a = a * b; }
inline bool operator>(Dual a, Dual b) { return a.v > b.v; }
inline bool operator<(Dual a, Dual b) { return a.v < b.v; }
inline Dual max0(Dual a) { return a.v > 0.0 ? a : Dual(0.0); }
inline Dual min0(Dual a) { return a.v < 0.0 ? a : Dual(0.0); }

int eps(int a, int b, int c) {
  if (a == b || b == c || a == c) return 0;
  // even permutations of (0,1,2)
  if ((a == 0 && b == 1 && c == 2) || (a == 1 && b == 2 && c == 0) || (a == 2 && b == 0 && c == 1)) return 1;
  return -1;
}

// The five stored components are xx, xy, xz, yy, yz; zz = -xx - yy.
template <typename R>
void q_full(const R* q5, long N, long s, M3<R> Q) {
  R xx = q5[0 * N + s], xy = q5[1 * N + s], xz = q5[2 * N + s];
  R yy = q5[3 * N + s], yz = q5[4 * N + s];
  Q[0][0] = xx; Q[0][1] = xy; Q[0][2] = xz;
  Q[1][0] = xy; Q[1][1] = yy; Q[1][2] = yz;
  Q[2][0] = xz; Q[2][1] = yz; Q[2][2] = -xx - yy;
}

template <typename R>
void q_store(const M3<R> Q, R* q5, long N, long s) {
  q5[0 * N + s] = Q[0][0]; q5[1 * N + s] = Q[0][1]; q5[2 * N + s] = Q[0][2];
  q5[3 * N + s] = Q[1][1]; q5[4 * N + s] = Q[1][2];
}

// Symmetric traceless projection.
template <typename R>
void sym_traceless(const M3<R> A, M3<R> out) {
  R tr = (A[0][0] + A[1][1] + A[2][2]) / 3.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) out[i][j] = 0.5 * (A[i][j] + A[j][i]) - (i == j ? tr : 0.0);
}

template <typename R>
void matmul(const M3<R> A, const M3<R> B, M3<R> C) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      R s = 0.0;
      for (int k = 0; k < 3; ++k) s += A[i][k] * B[k][j];
      C[i][j] = s;
    }
}

template <typename R>
R trace_prod(const M3<R> A, const M3<R> B) {  // tr(A B) = A_ij B_ji
  R s = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) s += A[i][j] * B[j][i];
  return s;
}

// Per-site stencil results (Sec. 3: finite differences on Q and psi).
template <typename R>
struct Derivs {
  R dQ[3][3][3];  // dQ[a][i][j] = d_a Q_ij
  R lapQ[3][3];
  R dpsi[3];
  R lappsi;
  R hpsi[3][3];
};

// Isotropic D3Q19 gradient 3 sum_i w_i c_ia f(x+c_i) and Laplacian 6 sum_i w_i (f(x+c_i)-f(x));
// Hessian of psi: three-point second difference on the diagonal, four corners off it.
template <typename R>
void derivs_at(const Box& B, const R* q5, const R* psi, int x, int y, int z, Derivs<R>& d) {
  long N = B.n();
  long s = B.at(x, y, z);
  M3<R> Q0;
  q_full(q5, N, s, Q0);
  R p0 = psi[s];
  d = Derivs<R>();
  for (int i = 1; i < NQ; ++i) {
    long n = B.at(x + CV[i][0], y + CV[i][1], z + CV[i][2]);
    M3<R> Qn;
    q_full(q5, N, n, Qn);
    R w = wgt(i);
    for (int a = 0; a < 3; ++a) {
      if (CV[i][a] == 0) continue;
      for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) d.dQ[a][p][q] += 3.0 * w * CV[i][a] * Qn[p][q];
      d.dpsi[a] += 3.0 * w * CV[i][a] * psi[n];
    }
    for (int p = 0; p < 3; ++p)
      for (int q = 0; q < 3; ++q) d.lapQ[p][q] += 6.0 * w * (Qn[p][q] - Q0[p][q]);
    d.lappsi += 6.0 * w * (psi[n] - p0);
  }
  for (int a = 0; a < 3; ++a) {
    int ea[3] = {0, 0, 0};
    ea[a] = 1;
    d.hpsi[a][a] = psi[B.at(x + ea[0], y + ea[1], z + ea[2])] - 2.0 * p0 +
                   psi[B.at(x - ea[0], y - ea[1], z - ea[2])];
    for (int b = 0; b < 3; ++b) {
      if (b == a) continue;
      int eb[3] = {0, 0, 0};
      eb[b] = 1;
      R spp = psi[B.at(x + ea[0] + eb[0], y + ea[1] + eb[1], z + ea[2] + eb[2])];
      R spm = psi[B.at(x + ea[0] - eb[0], y + ea[1] - eb[1], z + ea[2] - eb[2])];
      R smp = psi[B.at(x - ea[0] + eb[0], y - ea[1] + eb[1], z - ea[2] + eb[2])];
      R smm = psi[B.at(x - ea[0] - eb[0], y - ea[1] - eb[1], z - ea[2] - eb[2])];
      d.hpsi[a][b] = 0.25 * (spp - spm - smp + smm);
    }
  }
}

// Fourth-order central differences along the axes (radius 2):
//   d_a f   = [8 (f(+e_a) - f(-e_a)) - (f(+2e_a) - f(-2e_a))] / 12,
//   d_aa f  = [16 (f(+e_a) + f(-e_a)) - (f(+2e_a) + f(-2e_a)) - 30 f] / 12,
//   d_a d_b f (a != b) = d_a applied to d_b f (16 points),
// and the Laplacian as the sum of the three d_aa.
template <typename R, class G>
R r2_d1(const G& f, int a) {
  int e[3] = {0, 0, 0};
  e[a] = 1;
  return (8.0 * (f(e[0], e[1], e[2]) - f(-e[0], -e[1], -e[2])) -
          (f(2 * e[0], 2 * e[1], 2 * e[2]) - f(-2 * e[0], -2 * e[1], -2 * e[2]))) / 12.0;
}

template <typename R, class G>
R r2_d2(const G& f, int a) {
  int e[3] = {0, 0, 0};
  e[a] = 1;
  return (16.0 * (f(e[0], e[1], e[2]) + f(-e[0], -e[1], -e[2])) -
          (f(2 * e[0], 2 * e[1], 2 * e[2]) + f(-2 * e[0], -2 * e[1], -2 * e[2])) - 30.0 * f(0, 0, 0)) / 12.0;
}

template <typename R, class G>
R r2_mixed(const G& f, int a, int b) {
  const R c[5] = {1.0 / 12.0, -8.0 / 12.0, 0.0, 8.0 / 12.0, -1.0 / 12.0};  // weights of -2..2
  R s = 0.0;
  for (int i = -2; i <= 2; ++i)
    for (int j = -2; j <= 2; ++j) {
      if (i == 0 || j == 0) continue;
      int o[3] = {0, 0, 0};
      o[a] += i;
      o[b] += j;
      s += c[i + 2] * c[j + 2] * f(o[0], o[1], o[2]);
    }
  return s;
}

template <typename R>
void derivs_at_r2(const Box& B, const R* q5, const R* psi, int x, int y, int z, Derivs<R>& d) {
  long N = B.n();
  d = Derivs<R>();
  auto fpsi = [&](int dx, int dy, int dz) { return psi[B.at(x + dx, y + dy, z + dz)]; };
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < 3; ++q) {
      auto fq = [&](int dx, int dy, int dz) {
        M3<R> Qn;
        q_full(q5, N, B.at(x + dx, y + dy, z + dz), Qn);
        return Qn[p][q];
      };
      for (int a = 0; a < 3; ++a) {
        d.dQ[a][p][q] = r2_d1<R>(fq, a);
        d.lapQ[p][q] += r2_d2<R>(fq, a);
      }
    }
  for (int a = 0; a < 3; ++a) {
    d.dpsi[a] = r2_d1<R>(fpsi, a);
    d.lappsi += r2_d2<R>(fpsi, a);
    for (int b = 0; b < 3; ++b) d.hpsi[a][b] = (a == b) ? r2_d2<R>(fpsi, a) : r2_mixed<R>(fpsi, a, b);
  }
}

template <typename R>
void derivs_any(int stencil, const Box& B, const R* q5, const R* psi, int x, int y, int z, Derivs<R>& d) {
  if (stencil == 1) derivs_at_r2(B, q5, psi, x, y, z, d);
  else derivs_at(B, q5, psi, x, y, z, d);
}

// Local<R> quantities at one site: H (Eq. 2, Eq. 5), mu (Eq. 1, Eq. 5), free-energy density
// (Eq. 5) and the three parts of the stress (Eq. 3, Eq. 4).
template <typename R>
struct Local {
  M3<R> H;
  R mu;
  R fden;
  M3<R> sE;  // pressure + elastic + interfacial (Ericksen) stress
  M3<R> sR;  // reactive Beris-Edwards stress: flow-aligning xi terms + antisymmetric part
  M3<R> sA;  // active stress
};

template <typename R>
void local_at(const PR<R>& P, const M3<R> Q, R psi, const Derivs<R>& d, Local<R>& L) {
  const R chi = P.chi0 + P.chis * (1.0 + psi);
  M3<R> QQ;
  matmul(Q, Q, QQ);
  const R trQ2 = trace_prod(Q, Q);
  const R trQ3 = trace_prod(QQ, Q);
  // C_ab = eps_amn d_m Q_nb  (the curl of Q)
  M3<R> C;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      R s = 0.0;
      for (int m = 0; m < 3; ++m)
        for (int n = 0; n < 3; ++n) {
          int e = eps(a, m, n);
          if (e) s += e * d.dQ[m][n][b];
        }
      C[a][b] = s;
    }
  R g2 = d.dpsi[0] * d.dpsi[0] + d.dpsi[1] * d.dpsi[1] + d.dpsi[2] * d.dpsi[2];
  // -dF/dQ before projection
  M3<R> Hraw;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      R dij = (i == j) ? 1.0 : 0.0;
      Hraw[i][j] = -P.A0 * (1.0 - chi / 3.0) * Q[i][j] + P.A0 * chi * (QQ[i][j] - dij * trQ2 / 3.0) -
                   P.A0 * chi * trQ2 * Q[i][j] + P.K * d.lapQ[i][j] - 2.0 * P.K * P.q0 * (C[i][j] + C[j][i]) -
                   4.0 * P.K * P.q0 * P.q0 * Q[i][j] - P.W * (d.dpsi[i] * d.dpsi[j] - dij * g2 / 3.0);
    }
  sym_traceless(Hraw, L.H);

  // mu = dF/dpsi
  R divQ_dpsi = 0.0, Q_hess = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      divQ_dpsi += d.dQ[a][a][b] * d.dpsi[b];
      Q_hess += Q[a][b] * d.hpsi[a][b];
    }
  L.mu = -P.a * psi + P.b * psi * psi * psi - P.kphi * d.lappsi +
         P.A0 * P.chis * (-trQ2 / 6.0 - trQ3 / 3.0 + trQ2 * trQ2 / 4.0) - 2.0 * P.W * (divQ_dpsi + Q_hess);

  // free-energy density of Eq. 5
  R grad2 = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) grad2 += d.dQ[a][i][j] * d.dQ[a][i][j];
  R QC = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) QC += Q[i][j] * C[i][j];
  R anch = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) anch += d.dpsi[i] * Q[i][j] * d.dpsi[j];
  L.fden = -0.5 * P.a * psi * psi + 0.25 * P.b * psi * psi * psi * psi + 0.5 * P.kphi * g2 +
           P.A0 * (0.5 * (1.0 - chi / 3.0) * trQ2 - chi / 3.0 * trQ3 + chi / 4.0 * trQ2 * trQ2) +
           0.5 * P.K * grad2 + 2.0 * P.K * P.q0 * QC + 2.0 * P.K * P.q0 * P.q0 * trQ2 + P.W * anch;
  const R P0 = psi * L.mu - L.fden;

  // Pi_bgn = dF/d(d_b Q_gn) = K d_b Q_gn + 2 K q0 eps_mbg Q_mn
  R Pi[3][3][3];
  for (int b = 0; b < 3; ++b)
    for (int g = 0; g < 3; ++g)
      for (int n = 0; n < 3; ++n) {
        R s = P.K * d.dQ[b][g][n];
        for (int m = 0; m < 3; ++m) {
          int e = eps(m, b, g);
          if (e) s += 2.0 * P.K * P.q0 * e * Q[m][n];
        }
        Pi[b][g][n] = s;
      }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      R s = -(a == b ? P0 : 0.0);
      for (int g = 0; g < 3; ++g)
        for (int n = 0; n < 3; ++n) s -= d.dQ[a][g][n] * Pi[b][g][n];
      R Qdpsi = 0.0;
      for (int g = 0; g < 3; ++g) Qdpsi += Q[b][g] * d.dpsi[g];
      s -= d.dpsi[a] * (P.kphi * d.dpsi[b] + 2.0 * P.W * Qdpsi);
      L.sE[a][b] = s;
    }

  // reactive stress with Qt = Q + I/3
  M3<R> Qt;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Qt[i][j] = Q[i][j] + (i == j ? 1.0 / 3.0 : 0.0);
  M3<R> HQt, QtH, QH, HQ;
  matmul(L.H, Qt, HQt);
  matmul(Qt, L.H, QtH);
  matmul(Q, L.H, QH);
  matmul(L.H, Q, HQ);
  const R trQH = trace_prod(Q, L.H);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      L.sR[a][b] = -P.xi * HQt[a][b] - P.xi * QtH[a][b] + 2.0 * P.xi * Qt[a][b] * trQH + QH[a][b] - HQ[a][b];

  const R phic = 0.5 * (1.0 + psi);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) L.sA[a][b] = -P.zeta * phic * Q[a][b];
}

// Co-rotation term of Beris-Edwards (Eq. 2's strain-rotational part); Wg[a][b] = d_b u_a.
template <typename R>
void corotation(const M3<R> Wg, const M3<R> Q, R xi, M3<R> S) {
  M3<R> D, Om, Qt;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      D[i][j] = 0.5 * (Wg[i][j] + Wg[j][i]);
      Om[i][j] = 0.5 * (Wg[i][j] - Wg[j][i]);
      Qt[i][j] = Q[i][j] + (i == j ? 1.0 / 3.0 : 0.0);
    }
  M3<R> A, Bm;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      A[i][j] = xi * D[i][j] + Om[i][j];
      Bm[i][j] = xi * D[i][j] - Om[i][j];
    }
  M3<R> T1, T2;
  matmul(A, Qt, T1);
  matmul(Qt, Bm, T2);
  const R trQW = trace_prod(Q, Wg);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) S[i][j] = T1[i][j] + T2[i][j] - 2.0 * xi * Qt[i][j] * trQW;
}

// Isotropic gradient of a vector field at a site: Wg[a][b] = d_b u_a.
template <typename R>
void vec_grad_at(const Box& B, const R* u, int x, int y, int z, M3<R> Wg) {
  long N = B.n();
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) Wg[a][b] = 0.0;
  for (int i = 1; i < NQ; ++i) {
    long n = B.at(x + CV[i][0], y + CV[i][1], z + CV[i][2]);
    R w = wgt(i);
    for (int b = 0; b < 3; ++b) {
      if (CV[i][b] == 0) continue;
      for (int a = 0; a < 3; ++a) Wg[a][b] += 3.0 * w * CV[i][b] * u[a * N + n];
    }
  }
}

template <typename R>
void vec_grad_at_r2(const Box& B, const R* u, int x, int y, int z, M3<R> Wg) {
  long N = B.n();
  for (int a = 0; a < 3; ++a) {
    auto fu = [&](int dx, int dy, int dz) { return u[a * N + B.at(x + dx, y + dy, z + dz)]; };
    for (int b = 0; b < 3; ++b) Wg[a][b] = r2_d1<R>(fu, b);
  }
}

template <typename R>
void vec_grad_any(int stencil, const Box& B, const R* u, int x, int y, int z, M3<R> Wg) {
  if (stencil == 1) vec_grad_at_r2(B, u, x, y, z, Wg);
  else vec_grad_at(B, u, x, y, z, Wg);
}

template <typename R>
struct Work {
  std::vector<R> H, mu, sig, sigA, F, unew, fnew, rhsQ, rhsP, Qp, Pp;
};

// Stage 1-4 over the whole box: H (5), mu, total stress (9) per site.
template <typename R>
void fields_all(const Box& B, const PR<R>& P, const R* q5, const R* psi, R* H5, R* mu,
                R* sig9, R* sE9, R* sR9, R* sA9, R* fden) {
  long N = B.n();
#pragma omp parallel for schedule(static)
  for (int z = 0; z < B.nz; ++z)
    for (int y = 0; y < B.ny; ++y)
      for (int x = 0; x < B.nx; ++x) {
        long s = B.at(x, y, z);
        Derivs<R> d;
        derivs_any(P.stencil, B, q5, psi, x, y, z, d);
        M3<R> Q;
        q_full(q5, N, s, Q);
        Local<R> L;
        local_at(P, Q, psi[s], d, L);
        if (H5) q_store(L.H, H5, N, s);
        if (mu) mu[s] = L.mu;
        if (fden) fden[s] = L.fden;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) {
            int k = 3 * a + b;
            if (sig9) sig9[k * N + s] = L.sE[a][b] + L.sR[a][b] + L.sA[a][b];
            if (sE9) sE9[k * N + s] = L.sE[a][b];
            if (sR9) sR9[k * N + s] = L.sR[a][b];
            if (sA9) sA9[k * N + s] = L.sA[a][b];
          }
      }
}

// Stage 5: F_a = d_b sigma_ab with the isotropic gradient (stencil 0) or the fourth-order
// axis differences (stencil 1).
template <typename R>
void force_all(const Box& B, const R* sig9, R* F3, int stencil = 0) {
  long N = B.n();
#pragma omp parallel for schedule(static)
  for (int z = 0; z < B.nz; ++z)
    for (int y = 0; y < B.ny; ++y)
      for (int x = 0; x < B.nx; ++x) {
        long s = B.at(x, y, z);
        R F[3] = {0, 0, 0};
        if (stencil == 1) {
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
              auto fs = [&](int dx, int dy, int dz) { return sig9[(3 * a + b) * N + B.at(x + dx, y + dy, z + dz)]; };
              F[a] += r2_d1<R>(fs, b);
            }
          for (int a = 0; a < 3; ++a) F3[a * N + s] = F[a];
          continue;
        }
        for (int i = 1; i < NQ; ++i) {
          long n = B.at(x + CV[i][0], y + CV[i][1], z + CV[i][2]);
          R w = wgt(i);
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
              if (CV[i][b]) F[a] += 3.0 * w * CV[i][b] * sig9[(3 * a + b) * N + n];
        }
        for (int a = 0; a < 3; ++a) F3[a * N + s] = F[a];
      }
}

// Stage 6: BGK + Guo forcing (Eq. 7 as read), moments (Eq. 8), streaming (Eq. 6).
template <typename R>
void lb_all(const Box& B, const PR<R>& P, const R* f, const R* F3, R* fnew, R* unew) {
  long N = B.n();
  const LBSet L = lb_set(P.lattice);
  const R tau = P.tau;
#pragma omp parallel for schedule(static)
  for (int z = 0; z < B.nz; ++z)
    for (int y = 0; y < B.ny; ++y)
      for (int x = 0; x < B.nx; ++x) {
        long s = B.at(x, y, z);
        R rho = 0.0, j[3] = {0, 0, 0};
        for (int i = 0; i < L.q; ++i) {
          R fi = f[i * N + s];
          rho += fi;
          for (int a = 0; a < 3; ++a) j[a] += fi * L.c[i][a];
        }
        R F[3] = {F3[0 * N + s], F3[1 * N + s], F3[2 * N + s]};
        R u[3];
        for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * F[a]) / rho;
        R u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        for (int i = 0; i < L.q; ++i) {
          R cu = L.c[i][0] * u[0] + L.c[i][1] * u[1] + L.c[i][2] * u[2];
          R cF = L.c[i][0] * F[0] + L.c[i][1] * F[1] + L.c[i][2] * F[2];
          R uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
          R feq = L.w[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * u2);
          R Fi = (1.0 - 0.5 / tau) * L.w[i] * (3.0 * (cF - uF) + 9.0 * cu * cF);
          R fstar = f[i * N + s] - (f[i * N + s] - feq) / tau + Fi;
          long d = B.at(x + L.c[i][0], y + L.c[i][1], z + L.c[i][2]);
          fnew[i * N + d] = fstar;
        }
        for (int a = 0; a < 3; ++a) unew[a * N + s] = u[a];
      }
}

// Stage 6 in the form of Eqs. 9-11: the equilibrium carries the symmetric stress,
//   f_eq_i = w_i [rho + 3 rho c.u + (9/2)(c c - I/3) : (rho u u - sigma^S)],
// so that sum f_eq = rho, sum f_eq c = rho u and sum f_eq c c = rho/3 I + rho u u - sigma^S
// (Eq. 9 with the lattice pressure rho c_s^2 kept); the antisymmetric stress enters
// through F_i = 3 w_i c . FA, FA = div sigma^A, whose moments are 0, FA and 0 (Eq. 10).
// Collision f* = f - (f - f_eq)/tau + F_i (Eq. 7), rho u = sum f c (Eq. 8), streaming (Eq. 6).
template <typename R>
void lb_all_stress(const Box& B, const PR<R>& P, const R* f, const R* FA3, const R* sig9, R* fnew, R* unew) {
  long N = B.n();
  const LBSet L = lb_set(P.lattice);
  const R tau = P.tau;
#pragma omp parallel for schedule(static)
  for (int z = 0; z < B.nz; ++z)
    for (int y = 0; y < B.ny; ++y)
      for (int x = 0; x < B.nx; ++x) {
        long s = B.at(x, y, z);
        R rho = 0.0, j[3] = {0, 0, 0};
        for (int i = 0; i < L.q; ++i) {
          R fi = f[i * N + s];
          rho += fi;
          for (int a = 0; a < 3; ++a) j[a] += fi * L.c[i][a];
        }
        R u[3];
        for (int a = 0; a < 3; ++a) u[a] = j[a] / rho;
        // Pi = rho u u - sigma^S
        M3<R> Pi;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b)
            Pi[a][b] = rho * u[a] * u[b] - 0.5 * (sig9[(3 * a + b) * N + s] + sig9[(3 * b + a) * N + s]);
        R trPi = Pi[0][0] + Pi[1][1] + Pi[2][2];
        R FA[3] = {FA3[0 * N + s], FA3[1 * N + s], FA3[2 * N + s]};
        for (int i = 0; i < L.q; ++i) {
          R cu = L.c[i][0] * u[0] + L.c[i][1] * u[1] + L.c[i][2] * u[2];
          R cPc = 0.0;
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) cPc += L.c[i][a] * Pi[a][b] * L.c[i][b];
          R feq = L.w[i] * (rho + 3.0 * rho * cu + 4.5 * (cPc - trPi / 3.0));
          R cFA = L.c[i][0] * FA[0] + L.c[i][1] * FA[1] + L.c[i][2] * FA[2];
          R Fi = 3.0 * L.w[i] * cFA;
          R fstar = f[i * N + s] - (f[i * N + s] - feq) / tau + Fi;
          long d = B.at(x + L.c[i][0], y + L.c[i][1], z + L.c[i][2]);
          fnew[i * N + d] = fstar;
        }
        for (int a = 0; a < 3; ++a) unew[a * N + s] = u[a];
      }
}

// Stage 7 right-hand sides: -upwind advection + co-rotation + Gamma_Q H for Q;
// -div(upwind flux) + M lap mu for psi.
template <typename R>
void op_rhs(const Box& B, const PR<R>& P, const R* q5, const R* psi, const R* uadv,
            const R* H5, const R* mu, R* rq5, R* rp) {
  long N = B.n();
#pragma omp parallel for schedule(static)
  for (int z = 0; z < B.nz; ++z)
    for (int y = 0; y < B.ny; ++y)
      for (int x = 0; x < B.nx; ++x) {
        long s = B.at(x, y, z);
        int r[3] = {x, y, z};
        M3<R> Q, H, Wg, S;
        q_full(q5, N, s, Q);
        q_full(H5, N, s, H);
        vec_grad_any(P.stencil, B, uadv, x, y, z, Wg);
        corotation(Wg, Q, P.xi, S);
        M3<R> adv;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) adv[i][j] = 0.0;
        R div = 0.0;
        for (int a = 0; a < 3; ++a) {
          int rp1[3] = {r[0], r[1], r[2]}, rm1[3] = {r[0], r[1], r[2]};
          rp1[a] += 1;
          rm1[a] -= 1;
          long sp = B.at(rp1[0], rp1[1], rp1[2]);
          long sm = B.at(rm1[0], rm1[1], rm1[2]);
          R ua = uadv[a * N + s];
          M3<R> Qp, Qm;
          q_full(q5, N, sp, Qp);
          q_full(q5, N, sm, Qm);
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
              adv[i][j] += max0(ua) * (Q[i][j] - Qm[i][j]) + min0(ua) * (Qp[i][j] - Q[i][j]);
          // upwind face fluxes of psi at x + e_a/2 and x - e_a/2
          R ubp = 0.5 * (ua + uadv[a * N + sp]);
          R Jp = ubp * (ubp > 0.0 ? psi[s] : psi[sp]);
          R ubm = 0.5 * (uadv[a * N + sm] + ua);
          R Jm = ubm * (ubm > 0.0 ? psi[sm] : psi[s]);
          div += Jp - Jm;
        }
        R lapmu = 0.0;
        if (P.stencil == 1) {
          auto fm = [&](int dx, int dy, int dz) { return mu[B.at(x + dx, y + dy, z + dz)]; };
          for (int a = 0; a < 3; ++a) lapmu += r2_d2<R>(fm, a);
        } else {
          for (int i = 1; i < NQ; ++i) {
            long n = B.at(x + CV[i][0], y + CV[i][1], z + CV[i][2]);
            lapmu += 6.0 * wgt(i) * (mu[n] - mu[s]);
          }
        }
        M3<R> Rm;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) Rm[i][j] = -adv[i][j] + S[i][j] + P.gammaQ * H[i][j];
        // Q' = ST(Q + R) with ST the symmetric traceless projection; Q is already
        // symmetric traceless and ST is linear, so Q' = Q + ST(R).
        M3<R> Rp;
        sym_traceless(Rm, Rp);
        q_store(Rp, rq5, N, s);
        rp[s] = -div + P.M * lapmu;
      }
}

template <typename R>
void step_one(const Box& B, const PR<R>& P, R* f, R* q5, R* psi, R* uprev, Work<R>& w) {
  const long N = B.n();
  w.H.resize(5 * N); w.mu.resize(N); w.sig.resize(9 * N); w.F.resize(3 * N);
  const int q = lb_set(P.lattice).q;
  w.unew.resize(3 * N); w.fnew.resize(q * N); w.rhsQ.resize(5 * N); w.rhsP.resize(N);
  fields_all<R>(B, P, q5, psi, w.H.data(), w.mu.data(), w.sig.data(), nullptr, nullptr, nullptr, nullptr);
  if (P.lb_form == 1) {
    // force of the antisymmetric stress only; the symmetric part enters the equilibrium
    w.sigA.resize(9 * N);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        for (long k = 0; k < N; ++k)
          w.sigA[(3 * a + b) * N + k] = 0.5 * (w.sig[(3 * a + b) * N + k] - w.sig[(3 * b + a) * N + k]);
    force_all<R>(B, w.sigA.data(), w.F.data(), P.stencil);
    lb_all_stress<R>(B, P, f, w.F.data(), w.sig.data(), w.fnew.data(), w.unew.data());
  } else {
    force_all<R>(B, w.sig.data(), w.F.data(), P.stencil);
    lb_all<R>(B, P, f, w.F.data(), w.fnew.data(), w.unew.data());
  }
  const R* uadv = (P.coupling == 1) ? w.unew.data() : uprev;
  op_rhs<R>(B, P, q5, psi, uadv, w.H.data(), w.mu.data(), w.rhsQ.data(), w.rhsP.data());
  if (P.integrator == 1) {
    // Heun: predictor Q* = Q + R(Q), corrector Q' = Q + (R(Q) + R(Q*))/2, u held fixed.
    w.Qp.resize(5 * N); w.Pp.resize(N);
    for (long k = 0; k < 5 * N; ++k) w.Qp[k] = q5[k] + w.rhsQ[k];
    for (long k = 0; k < N; ++k) w.Pp[k] = psi[k] + w.rhsP[k];
    std::vector<R> H2(5 * N), mu2(N), rq2(5 * N), rp2(N);
    fields_all<R>(B, P, w.Qp.data(), w.Pp.data(), H2.data(), mu2.data(), nullptr, nullptr, nullptr, nullptr, nullptr);
    op_rhs<R>(B, P, w.Qp.data(), w.Pp.data(), uadv, H2.data(), mu2.data(), rq2.data(), rp2.data());
    for (long k = 0; k < 5 * N; ++k) q5[k] += 0.5 * (w.rhsQ[k] + rq2[k]);
    for (long k = 0; k < N; ++k) psi[k] += 0.5 * (w.rhsP[k] + rp2[k]);
  } else {
    for (long k = 0; k < 5 * N; ++k) q5[k] += w.rhsQ[k];
    for (long k = 0; k < N; ++k) psi[k] += w.rhsP[k];
  }
  std::memcpy(f, w.fnew.data(), sizeof(R) * q * N);
  std::memcpy(uprev, w.unew.data(), sizeof(R) * 3 * N);
}

// SplitMix64 (Steele, Lea & Flood 2014): the stream seeded with `seed` returns, at
// position k >= 1, mix(seed + k * 0x9E3779B97F4A7C15).
uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
  uint64_t z = seed + k * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

}  // namespace

extern "C" {

// D3Q19 table as used here (for index matching in tests).
// Threads the stage loops use (1 in the single-thread build).
int orc_num_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_lattice(int* c57, double* w19) {
  for (int i = 0; i < NQ; ++i) {
    for (int a = 0; a < 3; ++a) c57[3 * i + a] = CV[i][a];
    w19[i] = wgt(i);
  }
}

// The LB velocity set with q = 15 or 19 velocities (c: 3q ints, w: q doubles).
void orc_lattice_q(int q, int* c, double* w) {
  const LBSet L = lb_set(q);
  for (int i = 0; i < L.q; ++i) {
    for (int a = 0; a < 3; ++a) c[3 * i + a] = L.c[i][a];
    w[i] = L.w[i];
  }
}

// Uniform variate in [-1, 1) for (seed, instance, site, component): counter
// k = 1 + (instance << 40) + 5*site + component in the SplitMix64 stream of `seed`.
double orc_noise(uint64_t seed, int inst, long site, int comp) {
  uint64_t k = 1ULL + ((uint64_t)inst << 40) + 5ULL * (uint64_t)site + (uint64_t)comp;
  uint64_t r = splitmix64_at(seed, k);
  double u01 = (double)(r >> 11) * (1.0 / 9007199254740992.0);
  return 2.0 * u01 - 1.0;
}

// Initial state: rho = rho0, u = 0, psi = tanh((R - r)/2); inside r < R a cholesteric
// helix about z, n = (cos q0 (z - cz), sin q0 (z - cz), 0), Q = S0 (n n - I/3) plus
// noise * U[-1, 1) on each stored component; outside Q = 0.
void orc_init(int nx, int ny, int nz, const orc_params* P, uint64_t seed, int inst, double* f, double* q5,
              double* psi, double* u) {
  Box B{nx, ny, nz};
  long N = B.n();
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        long s = B.at(x, y, z);
        double dx = x - P->cx, dy = y - P->cy, dz = z - P->cz;
        double r = std::sqrt(dx * dx + dy * dy + dz * dz);
        psi[s] = std::tanh((P->R - r) / 2.0);
        M3<double> Q;
        std::memset(Q, 0, sizeof(Q));
        if (r < P->R) {
          double n[3] = {std::cos(P->q0 * dz), std::sin(P->q0 * dz), 0.0};
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) Q[i][j] = P->S0 * (n[i] * n[j] - (i == j ? 1.0 / 3.0 : 0.0));
        }
        q_store(Q, q5, N, s);
        if (r < P->R) {
          for (int c = 0; c < 5; ++c) q5[c * N + s] += P->noise * orc_noise(seed, inst, s, c);
        }
        const LBSet L = lb_set(P->lattice);
        for (int i = 0; i < L.q; ++i) f[i * N + s] = L.w[i] * P->rho0;
        for (int a = 0; a < 3; ++a) u[a * N + s] = 0.0;
      }
}

// Stages 1-4 over the box.  Any output pointer may be null.
void orc_fields(int nx, int ny, int nz, const orc_params* P, const double* q5, const double* psi, double* H5,
                double* mu, double* sig9, double* sE9, double* sR9, double* sA9, double* fden) {
  Box B{nx, ny, nz};
  fields_all<double>(B, promote<double>(*P), q5, psi, H5, mu, sig9, sE9, sR9, sA9, fden);
}

void orc_force(int nx, int ny, int nz, const double* sig9, double* F3) {
  Box B{nx, ny, nz};
  force_all(B, sig9, F3);
}

void orc_force_st(int stencil, int nx, int ny, int nz, const double* sig9, double* F3) {
  Box B{nx, ny, nz};
  force_all(B, sig9, F3, stencil);
}

// Stencils (0 = isotropic radius 1, 1 = fourth-order radius 2) on a scalar field.
void orc_stencils_st(int stencil, int nx, int ny, int nz, const double* s, double* grad3, double* lap,
                     double* hess9) {
  Box B{nx, ny, nz};
  long N = B.n();
  std::vector<double> zero(5 * N, 0.0);
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        long k = B.at(x, y, z);
        Derivs<double> d;
        derivs_any(stencil, B, zero.data(), s, x, y, z, d);
        for (int a = 0; a < 3; ++a) grad3[a * N + k] = d.dpsi[a];
        lap[k] = d.lappsi;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) hess9[(3 * a + b) * N + k] = d.hpsi[a][b];
      }
}

// Stencils on a scalar field (for the stencil pins).
void orc_stencils(int nx, int ny, int nz, const double* s, double* grad3, double* lap, double* hess9) {
  Box B{nx, ny, nz};
  long N = B.n();
  std::vector<double> zero(5 * N, 0.0);
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        long k = B.at(x, y, z);
        Derivs<double> d;
        derivs_at(B, zero.data(), s, x, y, z, d);
        for (int a = 0; a < 3; ++a) grad3[a * N + k] = d.dpsi[a];
        lap[k] = d.lappsi;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) hess9[(3 * a + b) * N + k] = d.hpsi[a][b];
      }
}

// Per-site co-rotation S(W, Q) (full 3x3 in and out; Wg[a][b] = d_b u_a).
void orc_corotation(const double* Wg9, const double* Q9, double xi, double* S9) {
  M3<double> W, Q, S;
  for (int i = 0; i < 9; ++i) { W[i / 3][i % 3] = Wg9[i]; Q[i / 3][i % 3] = Q9[i]; }
  corotation(W, Q, xi, S);
  for (int i = 0; i < 9; ++i) S9[i] = S[i / 3][i % 3];
}

// Per-site Q update pieces over the box for a given advecting velocity: the projected
// right-hand sides of Q (5) and psi (1), and the velocity gradient W (9).
void orc_op_rhs(int nx, int ny, int nz, const orc_params* P, const double* q5, const double* psi,
                const double* uadv, const double* H5, const double* mu, double* rq5, double* rp, double* W9) {
  Box B{nx, ny, nz};
  op_rhs<double>(B, promote<double>(*P), q5, psi, uadv, H5, mu, rq5, rp);
  if (W9) {
    long N = B.n();
    for (int z = 0; z < nz; ++z)
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          long s = B.at(x, y, z);
          M3<double> Wg;
          vec_grad_any(P->stencil, B, uadv, x, y, z, Wg);
          for (int k = 0; k < 9; ++k) W9[k * N + s] = Wg[k / 3][k % 3];
        }
  }
}

// nsteps full hybrid steps in place.  f: 19*N pre-collision populations (unshifted),
// q5: 5*N, psi: N, uprev: 3*N = u of the previous step (0 at t = 0).
void orc_step(int nx, int ny, int nz, const orc_params* P, double* f, double* q5, double* psi, double* uprev,
              long nsteps) {
  Box B{nx, ny, nz};
  Work<double> w;
  for (long t = 0; t < nsteps; ++t) step_one<double>(B, promote<double>(*P), f, q5, psi, uprev, w);
}

// Stage 6 alone (for LB pins): collide with a given force and stream.
void orc_lb(int nx, int ny, int nz, const orc_params* P, const double* f, const double* F3, double* fnew,
            double* unew) {
  Box B{nx, ny, nz};
  lb_all<double>(B, promote<double>(*P), f, F3, fnew, unew);
}

// Stage 6 in the form of Eqs. 9-11 alone: FA3 = force of the antisymmetric stress, sig9 =
// the stress whose symmetric part enters the equilibrium.
void orc_lb_stress(int nx, int ny, int nz, const orc_params* P, const double* f, const double* FA3,
                   const double* sig9, double* fnew, double* unew) {
  Box B{nx, ny, nz};
  lb_all_stress<double>(B, promote<double>(*P), f, FA3, sig9, fnew, unew);
}

// Conserved sums and centroid moments (FP64):
// out[0] = sum rho, out[1] = sum psi, out[2..4] = sum_i f_i c_i, out[5..7] = sum phi_c cos(2 pi x_a/L_a),
// out[8..10] = sum phi_c sin(2 pi x_a/L_a), out[11] = sum phi_c; phi_c = (1 + psi)/2.
void orc_observables_q(int q, int nx, int ny, int nz, const double* f, const double* psi, double* out) {
  Box B{nx, ny, nz};
  const LBSet V = lb_set(q);
  long N = B.n();
  for (int k = 0; k < 12; ++k) out[k] = 0.0;
  const double PI = 3.14159265358979323846;
  int L[3] = {nx, ny, nz};
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        long s = B.at(x, y, z);
        for (int i = 0; i < V.q; ++i) {
          double fi = f[i * N + s];
          out[0] += fi;
          for (int a = 0; a < 3; ++a) out[2 + a] += fi * V.c[i][a];
        }
        out[1] += psi[s];
        double pc = 0.5 * (1.0 + psi[s]);
        int r[3] = {x, y, z};
        for (int a = 0; a < 3; ++a) {
          out[5 + a] += pc * std::cos(2.0 * PI * r[a] / L[a]);
          out[8 + a] += pc * std::sin(2.0 * PI * r[a] / L[a]);
        }
        out[11] += pc;
      }
}

void orc_observables(int nx, int ny, int nz, const double* f, const double* psi, double* out) {
  orc_observables_q(19, nx, ny, nz, f, psi, out);
}

// Forward-mode tangent of nsteps steps.  (f, q5, psi, u) and their tangents (df, dq5,
// dpsi, du) advance together; the parameters zeta and q0 carry the tangents dzeta and dq0,
// all other parameters are fixed.  Used as an independent derivative for the adjoint.
void orc_step_tangent(int nx, int ny, int nz, const orc_params* P, double dzeta, double dq0, double* f,
                      double* df, double* q5, double* dq5, double* psi, double* dpsi, double* u, double* du,
                      long nsteps) {
  Box B{nx, ny, nz};
  const long N = B.n();
  const long q = lb_set(P->lattice).q;
  std::vector<Dual> F(q * N), Q(5 * N), S(N), U(3 * N);
  for (long k = 0; k < q * N; ++k) F[k] = Dual(f[k], df[k]);
  for (long k = 0; k < 5 * N; ++k) Q[k] = Dual(q5[k], dq5[k]);
  for (long k = 0; k < N; ++k) S[k] = Dual(psi[k], dpsi[k]);
  for (long k = 0; k < 3 * N; ++k) U[k] = Dual(u[k], du[k]);
  PR<Dual> pr = promote<Dual>(*P);
  pr.zeta.d = dzeta;
  pr.q0.d = dq0;
  Work<Dual> w;
  for (long t = 0; t < nsteps; ++t) step_one<Dual>(B, pr, F.data(), Q.data(), S.data(), U.data(), w);
  for (long k = 0; k < q * N; ++k) { f[k] = F[k].v; df[k] = F[k].d; }
  for (long k = 0; k < 5 * N; ++k) { q5[k] = Q[k].v; dq5[k] = Q[k].d; }
  for (long k = 0; k < N; ++k) { psi[k] = S[k].v; dpsi[k] = S[k].d; }
  for (long k = 0; k < 3 * N; ++k) { u[k] = U[k].v; du[k] = U[k].d; }
}

}  // extern "C"
