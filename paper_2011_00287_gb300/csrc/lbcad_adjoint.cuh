// lbcad_adjoint.cuh -- reverse mode (vector-Jacobian products) of one hybrid step.
//
// The step maps the stored state s_t = (g*, Q, psi, u) to s_{t+1}.  Given the cotangent
// lam_{t+1} of s_{t+1}, four gather-form kernels produce lam_t:
//   RK1 k_adj_update : per site, VJP of update_math (upwind/co-rotation Q update,
//                      Cahn-Hilliard psi update, BGK + Guo collision) with respect to its
//                      88 inputs (F, lap mu, grad u, Q and psi faces, u faces, H, pulled g),
//                      by a hand-written reverse sweep (update_math_vjp)
//   RK2 k_adj_spread : transposes of the stencils that fed update_math: div sigma -> sigma,
//                      lap mu -> mu, grad u -> u, face reads -> Q/psi/u, the pull -> g*
//   RK3 k_adj_fields : per site, VJP of local_fields (H, mu, sigma of Eqs. 2-5) with respect
//                      to its 36 inputs (Q, psi and their stencils) and to zeta and q0
//   RK4 k_adj_gather : transposes of the Q/psi stencils (gradient, Laplacian, Hessian)
// The VJP of local_fields runs the forward device function on dual numbers carrying K
// tangents (forward mode, K input directions per pass), so it differentiates exactly the
// arithmetic the step executes.  Stencil transposes use the negated offsets on the
// periodic lattice, so no site is written by two threads.
#pragma once

#include "lbcad_kernels.cuh"

namespace lbcad {

// ---------------------------------------------------------------- dual numbers
template <typename S, int K>
struct Dual {
  S v;
  S d[K];
  __device__ __forceinline__ Dual() {}
  __device__ __forceinline__ Dual(S x) : v(x) {
#pragma unroll
    for (int k = 0; k < K; ++k) d[k] = S(0);
  }
};

template <typename S, int K>
__device__ __forceinline__ Dual<S, K> operator+(const Dual<S, K>& a, const Dual<S, K>& b) {
  Dual<S, K> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
template <typename S, int K>
__device__ __forceinline__ Dual<S, K> operator-(const Dual<S, K>& a, const Dual<S, K>& b) {
  Dual<S, K> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
template <typename S, int K>
__device__ __forceinline__ Dual<S, K> operator-(const Dual<S, K>& a) {
  Dual<S, K> r;
  r.v = -a.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = -a.d[k];
  return r;
}
template <typename S, int K>
__device__ __forceinline__ Dual<S, K> operator*(const Dual<S, K>& a, const Dual<S, K>& b) {
  Dual<S, K> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
  return r;
}
template <typename S, int K>
__device__ __forceinline__ Dual<S, K> operator/(const Dual<S, K>& a, const Dual<S, K>& b) {
  Dual<S, K> r;
  const S inv = S(1) / b.v;
  r.v = a.v * inv;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * inv;
  return r;
}
template <typename S, int K>
__device__ __forceinline__ Dual<S, K>& operator+=(Dual<S, K>& a, const Dual<S, K>& b) {
  a = a + b;
  return a;
}
template <typename S, int K>
__device__ __forceinline__ Dual<S, K>& operator-=(Dual<S, K>& a, const Dual<S, K>& b) {
  a = a - b;
  return a;
}
template <typename S, int K>
__device__ __forceinline__ bool operator>(const Dual<S, K>& a, const Dual<S, K>& b) { return a.v > b.v; }
template <typename S, int K>
__device__ __forceinline__ bool operator<(const Dual<S, K>& a, const Dual<S, K>& b) { return a.v < b.v; }

template <typename S, int K>
__device__ __forceinline__ Coef<Dual<S, K>> dual_coef(const Coef<S>& c) {
  Coef<Dual<S, K>> r;
  r.tau_inv = c.tau_inv; r.guo = c.guo; r.rho0 = c.rho0;
  r.A0 = c.A0; r.chi0 = c.chi0; r.chis = c.chis; r.K = c.K; r.q0 = c.q0; r.gammaQ = c.gammaQ; r.xi = c.xi;
  r.a = c.a; r.b = c.b; r.kphi = c.kphi; r.M = c.M; r.W = c.W; r.zeta = c.zeta;
  return r;
}

// Buffers of one reverse step (all [component][site]).
template <typename T>
struct AdjDesc {
  InstDesc<T> I;      // state s_t in I.*_in, its sigma/mu/H in I.sig/mu/H; *_out unused
  const T* lg;        // cotangent of s_{t+1}: g* (19), Q (5), psi (1), u (3)
  const T* lq;
  const T* lp;
  const T* lu;
  T* A;               // RK1 output: 88 input cotangents of update_math per site
  T* Bf;              // RK3 output: 36 input cotangents of local_fields per site
  T* ls;              // RK2 output: cotangents of sigma (9), mu (1), H (5)
  T* og;              // cotangent of s_t: g* (19), Q (5), psi (1), u (3)
  T* oq;
  T* op;
  T* ou;
  double* pgrad;      // per-block partial sums of d/dzeta, d/dq0 (2 per block)
};

constexpr int kAdjBlock = 128;

// ---------------------------------------------------------------- reverse mode of update_math
// Vector-Jacobian product of update_math (D3Q19 body-force collision, Euler update) at one
// site, by a hand-written reverse sweep over the forward arithmetic: in = the 88 inputs
// (layout of k_adj_update), lo = the cotangents of the 28 outputs (qn 0-4, pn 5, u 6-8,
// g 9-27), out = the cotangents of the 88 inputs.  The branches (upwind selection, face
// fluxes) take the side the forward takes, as forward-mode differentiation of the same
// code would.
template <typename T, bool SHIFT>
__device__ __forceinline__ void update_math_vjp(const Coef<T>& c, const T in[88], const T lo[28], T out[88]) {
  const T* F = in;
  const T lapmu_unused = in[3];
  (void)lapmu_unused;
  T W[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) W[a][b] = in[4 + 3 * a + b];
  const T* q0 = in + 13;
  const T* qfl = in + 18;  // qf[f][k] = qfl[5 f + k]
  const T p0 = in[48];
  const T* pf = in + 49;
  const T* u0 = in + 55;
  const T* uf = in + 58;
  const T* g = in + 69;
#pragma unroll
  for (int j = 0; j < 88; ++j) out[j] = T(0);

  // ---- LB collision (outputs u 6-8, g 9-27)
  T m0 = g[0];
  T jm[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int i = 1; i < 19; i += 2) {
    m0 += g[i] + g[i + 1];
    const T dg = g[i] - g[i + 1];
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (lat_c(i, a)) jm[a] += lat_c(i, a) > 0 ? dg : -dg;
  }
  const T rho = SHIFT ? (c.rho0 + m0) : m0;
  const T rinv = T(1) / rho;
  T u[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) u[a] = (jm[a] + T(0.5) * F[a]) * rinv;
  const T u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const T r45 = T(4.5) * rho, r3 = T(3) * rho, om = c.tau_inv;
  T lu[3] = {lo[6], lo[7], lo[8]};
  T lF[3] = {T(0), T(0), T(0)};
  T lbase = T(0), lr45 = T(0), lr3 = T(0), luF = T(0);
  {
    const T w = T(lat_w(0));
    const T l0 = lo[9];
    out[69] += (T(1) - om) * l0;
    lbase += om * w * l0;
    luF += -T(3) * c.guo * w * l0;
  }
#pragma unroll
  for (int i = 1; i < 19; i += 2) {
    const T w = T(lat_w(i)), gw = c.guo * w;
    const T cu = T(lat_c(i, 0)) * u[0] + T(lat_c(i, 1)) * u[1] + T(lat_c(i, 2)) * u[2];
    const T cF = T(lat_c(i, 0)) * F[0] + T(lat_c(i, 1)) * F[1] + T(lat_c(i, 2)) * F[2];
    const T lp = lo[9 + i], lm = lo[10 + i];
    out[69 + i] += (T(1) - om) * lp;
    out[70 + i] += (T(1) - om) * lm;
    const T lA = om * (lp + lm), lB = om * (lp - lm), lC = lp + lm, lE = lp - lm;
    lbase += w * lA;
    lr45 += w * cu * cu * lA;
    lr3 += w * cu * lB;
    luF += -T(3) * gw * lC;
    const T lcu = T(2) * w * r45 * cu * lA + w * r3 * lB + T(9) * gw * cF * lC;
    const T lcF = T(9) * gw * cu * lC + T(3) * gw * lE;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (lat_c(i, a)) {
        lu[a] += T(lat_c(i, a)) * lcu;
        lF[a] += T(lat_c(i, a)) * lcF;
      }
    }
  }
  // base = m0 - 1.5 rho u2 (shifted) or rho - 1.5 rho u2; r45 = 4.5 rho; r3 = 3 rho
  T lm0 = T(0), lrho = T(0), lu2 = T(0);
  if (SHIFT) lm0 += lbase; else lrho += lbase;
  lrho += -T(1.5) * u2 * lbase + T(4.5) * lr45 + T(3) * lr3;
  lu2 += -T(1.5) * rho * lbase;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lu[a] += T(2) * u[a] * lu2 + F[a] * luF;
    lF[a] += u[a] * luF;
  }
  // u = (j + F/2) / rho
  T lrinv = T(0), lj[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lrinv += (jm[a] + T(0.5) * F[a]) * lu[a];
    lj[a] = rinv * lu[a];
    lF[a] += T(0.5) * rinv * lu[a];
  }
  lrho += -rinv * rinv * lrinv;
  lm0 += lrho;
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    T v = lm0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (lat_c(i, a)) v += T(lat_c(i, a)) * lj[a];
    out[69 + i] += v;
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) out[a] += lF[a];

  // ---- order-parameter update (outputs qn 0-4, pn 5)
  const T xi = c.xi;
  T lq0[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    lq0[k] = lo[k];
    out[64 + k] += c.gammaQ * lo[k];
  }
  out[48] += lo[5];              // p0
  out[3] += c.M * lo[5];         // lap mu
  const T ldivJ = -lo[5];
  // co-rotation S of the five stored components
  T Q[3][3];
  full3(q0, Q);
  T Dm[3][3], Om[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Dm[i][j] = T(0.5) * (W[i][j] + W[j][i]);
      Om[i][j] = T(0.5) * (W[i][j] - W[j][i]);
    }
  T trQW = T(0);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) trQW += Q[i][j] * W[j][i];
  const T cq = -T(2) * xi * trQW;
  const T c23 = T(2) * xi / T(3);
  T lQ[3][3], lD[3][3], lO[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) lQ[i][j] = lD[i][j] = lO[i][j] = T(0);
  T lcq = T(0), lcdiag = T(0);
  const int I5[5] = {0, 0, 0, 1, 1};
  const int J5[5] = {0, 1, 2, 1, 2};
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int i = I5[k], j = J5[k];
    const T L = lo[k];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      lD[i][m] += xi * L * Q[m][j];
      lQ[m][j] += xi * L * Dm[i][m];
      lQ[i][m] += xi * L * Dm[m][j];
      lD[m][j] += xi * L * Q[i][m];
      lO[i][m] += L * Q[m][j];
      lQ[m][j] += L * Om[i][m];
      lQ[i][m] -= L * Om[m][j];
      lO[m][j] -= L * Q[i][m];
    }
    lD[i][j] += c23 * L;
    lcq += L * Q[i][j];
    lQ[i][j] += cq * L;
    if (i == j) lcdiag += L;
  }
  // cdiag = cq/3 - (2 xi/9) trD; cq = -2 xi tr(QW)
  lcq += lcdiag / T(3);
  const T ltrD = -(T(2) * xi / T(9)) * lcdiag;
  const T ltrQW = -T(2) * xi * lcq;
  T lW[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) lW[i][j] = T(0);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    lD[i][i] += ltrD;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      lQ[i][j] += W[j][i] * ltrQW;
      lW[j][i] += Q[i][j] * ltrQW;
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      lW[i][j] += T(0.5) * (lD[i][j] + lO[i][j]);
      lW[j][i] += T(0.5) * (lD[i][j] - lO[i][j]);
    }
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) out[4 + 3 * a + b] += lW[a][b];
  lq0[0] += lQ[0][0] - lQ[2][2];
  lq0[1] += lQ[0][1] + lQ[1][0];
  lq0[2] += lQ[0][2] + lQ[2][0];
  lq0[3] += lQ[1][1] - lQ[2][2];
  lq0[4] += lQ[1][2] + lQ[2][1];
  // upwind advection of Q and the psi face fluxes
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int ip = 2 * a, im = 2 * a + 1;
    const T up = u0[a] > T(0) ? u0[a] : T(0);
    const T um = u0[a] < T(0) ? u0[a] : T(0);
    T lup = T(0), lum = T(0);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const T ladv = -lo[k];
      lup += (q0[k] - qfl[5 * im + k]) * ladv;
      lum += (qfl[5 * ip + k] - q0[k]) * ladv;
      lq0[k] += (up - um) * ladv;
      out[18 + 5 * im + k] += -up * ladv;
      out[18 + 5 * ip + k] += um * ladv;
    }
    T lu0 = (u0[a] > T(0) ? lup : T(0)) + (u0[a] < T(0) ? lum : T(0));
    const T ubp = T(0.5) * (u0[a] + uf[ip]);
    const T lJp = ldivJ;
    if (ubp > T(0)) out[48] += ubp * lJp; else out[49 + ip] += ubp * lJp;
    const T lubp = (ubp > T(0) ? p0 : pf[ip]) * lJp;
    lu0 += T(0.5) * lubp;
    out[58 + ip] += T(0.5) * lubp;
    const T ubm = T(0.5) * (uf[im] + u0[a]);
    const T lJm = -ldivJ;
    if (ubm > T(0)) out[49 + im] += ubm * lJm; else out[48] += ubm * lJm;
    const T lubm = (ubm > T(0) ? pf[im] : p0) * lJm;
    out[58 + im] += T(0.5) * lubm;
    lu0 += T(0.5) * lubm;
    out[55 + a] += lu0;
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) out[13 + k] += lq0[k];
}

// ---------------------------------------------------------------- RK1
template <typename T, bool SHIFT>
__global__ void __launch_bounds__(kAdjBlock) k_adj_update(AdjDesc<T> A) {
  const InstDesc<T>& I = A.I;
  const long long N = I.N;
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  const int nx = I.nx, ny = I.ny, nz = I.nz;
  const int x = (int)(s % nx);
  const long long t = s / nx;
  const int y = (int)(t % ny), z = (int)(t / ny);
  GlobalAcc<T> acc;
  acc.q_ = I.q_in; acc.ps = I.psi_in; acc.sg = I.sig; acc.mu_ = I.mu; acc.u_ = I.u_in;
  acc.N = N;
  acc.nb = make_nbr(x, y, z, nx, ny, nz);
  // forward inputs of update_math, packed: F 0-2, lapmu 3, Wg 4-12, q0 13-17, qf 18-47,
  // p0 48, pf 49-54, u0 55-57, uf 58-63, Hs 64-68, g 69-87
  T in[88];
  {
    T F[3], lapmu, Wg[3][3], q0[5], qf[6][5], p0, pf[6], u0[3], uf[6];
    gather_update<T>(acc, F, lapmu, Wg, q0, qf, p0, pf, u0, uf);
    for (int a = 0; a < 3; ++a) in[a] = F[a];
    in[3] = lapmu;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) in[4 + 3 * a + b] = Wg[a][b];
    for (int k = 0; k < 5; ++k) in[13 + k] = q0[k];
    for (int f = 0; f < 6; ++f)
      for (int k = 0; k < 5; ++k) in[18 + 5 * f + k] = qf[f][k];
    in[48] = p0;
    for (int f = 0; f < 6; ++f) in[49 + f] = pf[f];
    for (int a = 0; a < 3; ++a) in[55 + a] = u0[a];
    for (int f = 0; f < 6; ++f) in[58 + f] = uf[f];
    for (int k = 0; k < 5; ++k) in[64 + k] = I.H[k * N + s];
    for (int i = 0; i < 19; ++i) in[69 + i] = I.g_in[i * N + acc.nb.off(-lat_c(i, 0), -lat_c(i, 1), -lat_c(i, 2))];
  }
  // output cotangents: qn 0-4, pn 5, u 6-8, g 9-27
  T lo[28];
  for (int k = 0; k < 5; ++k) lo[k] = A.lq[k * N + s];
  lo[5] = A.lp[s];
  for (int a = 0; a < 3; ++a) lo[6 + a] = A.lu[a * N + s];
  for (int i = 0; i < 19; ++i) lo[9 + i] = A.lg[i * N + s];
  T ci[88];
  update_math_vjp<T, SHIFT>(I.c, in, lo, ci);
  for (int j = 0; j < 88; ++j) A.A[j * N + s] = ci[j];
}

// ---------------------------------------------------------------- RK2
// Transposes of the stencils of gather_update and of the pull, gathered at site y.
template <typename T>
__global__ void __launch_bounds__(kAdjBlock) k_adj_spread(AdjDesc<T> A) {
  const InstDesc<T>& I = A.I;
  const long long N = I.N;
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  const int nx = I.nx, ny = I.ny, nz = I.nz;
  const int x = (int)(s % nx);
  const long long t = s / nx;
  const int y = (int)(t % ny), z = (int)(t / ny);
  const Nbr nb = make_nbr(x, y, z, nx, ny, nz);
  const T* __restrict__ a = A.A;
  // F_a(x) = sum_b sum_{i odd, c_ib != 0} sgn(c_ib) wt_i (sigma_ab(x + c_i) - sigma_ab(x - c_i))
  T ls[9];
  for (int k = 0; k < 9; ++k) ls[k] = T(0);
  T lu[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int i = 1; i < 19; i += 2) {
    const int cx = lat_c(i, 0), cy = lat_c(i, 1), cz = lat_c(i, 2);
    const T wt = lat_c2(i) == 1 ? T(2.0 / 12.0) : T(1.0 / 12.0);
    const long long m = nb.off(-cx, -cy, -cz);  // y - c_i
    const long long p = nb.off(cx, cy, cz);     // y + c_i
    const int cc[3] = {cx, cy, cz};
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (cc[b] == 0) continue;
      const T w = cc[b] > 0 ? wt : -wt;
#pragma unroll
      for (int aa = 0; aa < 3; ++aa) {
        ls[3 * aa + b] += w * (a[aa * N + m] - a[aa * N + p]);                       // F
        lu[aa] += w * (a[(4 + 3 * aa + b) * N + m] - a[(4 + 3 * aa + b) * N + p]);  // grad u
      }
    }
  }
  // lap mu(x) = sum_i lw_i mu(x + c_i) - 4 mu(x): symmetric
  T lmu = -T(4) * a[3 * N + s];
#pragma unroll
  for (int i = 1; i < 19; ++i) {
    const T lw = lat_c2(i) == 1 ? T(1.0 / 3.0) : T(1.0 / 6.0);
    lmu += lw * a[3 * N + nb.off(-lat_c(i, 0), -lat_c(i, 1), -lat_c(i, 2))];
  }
  for (int k = 0; k < 9; ++k) A.ls[k * N + s] = ls[k];
  A.ls[9 * N + s] = lmu;
  for (int k = 0; k < 5; ++k) A.ls[(10 + k) * N + s] = a[(64 + k) * N + s];
  // face reads: qf[f](x) = q(x + c_{f+1}), uf[2a](x) = u_a(x + e_a), uf[2a+1](x) = u_a(x - e_a)
  T lq[5], lp = a[48 * N + s];
  for (int k = 0; k < 5; ++k) lq[k] = a[(13 + k) * N + s];
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    const int i = f + 1;
    const long long m = nb.off(-lat_c(i, 0), -lat_c(i, 1), -lat_c(i, 2));
#pragma unroll
    for (int k = 0; k < 5; ++k) lq[k] += a[(18 + 5 * f + k) * N + m];
    lp += a[(49 + f) * N + m];
  }
#pragma unroll
  for (int aa = 0; aa < 3; ++aa) {
    lu[aa] += a[(55 + aa) * N + s];
    const int ip = 1 + 2 * aa, im = 2 + 2 * aa;  // +e_a, -e_a
    lu[aa] += a[(58 + 2 * aa) * N + nb.off(-lat_c(ip, 0), -lat_c(ip, 1), -lat_c(ip, 2))];
    lu[aa] += a[(59 + 2 * aa) * N + nb.off(-lat_c(im, 0), -lat_c(im, 1), -lat_c(im, 2))];
  }
  for (int k = 0; k < 5; ++k) A.oq[k * N + s] = lq[k];
  A.op[s] = lp;
  for (int aa = 0; aa < 3; ++aa) A.ou[aa * N + s] = lu[aa];
  // pull: g[i](x) = g*_i(x - c_i)  =>  lam g*_i(y) = lam g[i](y + c_i)
#pragma unroll
  for (int i = 0; i < 19; ++i) A.og[i * N + s] = a[(69 + i) * N + nb.off(lat_c(i, 0), lat_c(i, 1), lat_c(i, 2))];
}

// ---------------------------------------------------------------- RK3
// Inputs of local_fields, packed: q0 0-4, p0 5, dq 6-20 (a*5 + k), lapq 21-25, dp 26-28,
// lapp 29, hp 30-35; two more tangent directions: zeta (36), q0 parameter (37).
template <typename T, int K>
__global__ void __launch_bounds__(kAdjBlock) k_adj_fields(AdjDesc<T> A) {
  const InstDesc<T>& I = A.I;
  const long long N = I.N;
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double pz = 0.0, pq = 0.0;
  if (s < N) {
    const int nx = I.nx, ny = I.ny, nz = I.nz;
    const int x = (int)(s % nx);
    const long long t = s / nx;
    const int y = (int)(t % ny), z = (int)(t / ny);
    GlobalAcc<T> acc;
    acc.q_ = I.q_in; acc.ps = I.psi_in; acc.N = N;
    acc.nb = make_nbr(x, y, z, nx, ny, nz);
    T in[36];
    {
      T q0[5], p0, dq[3][5], lapq[5], dp[3], lapp, hp[6];
      gather_fields<T>(acc, q0, p0, dq, lapq, dp, lapp, hp);
      for (int k = 0; k < 5; ++k) in[k] = q0[k];
      in[5] = p0;
      for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 5; ++k) in[6 + 5 * a + k] = dq[a][k];
      for (int k = 0; k < 5; ++k) in[21 + k] = lapq[k];
      for (int a = 0; a < 3; ++a) in[26 + a] = dp[a];
      in[29] = lapp;
      for (int k = 0; k < 6; ++k) in[30 + k] = hp[k];
    }
    // output cotangents: H 0-4, mu 5, sigma 6-14
    T lo[15];
    for (int k = 0; k < 5; ++k) lo[k] = A.ls[(10 + k) * N + s];
    lo[5] = A.ls[9 * N + s];
    for (int k = 0; k < 9; ++k) lo[6 + k] = A.ls[k * N + s];
    for (int j0 = 0; j0 < 38; j0 += K) {
      using D = Dual<T, K>;
      Coef<D> cd = dual_coef<T, K>(I.c);
      if (36 >= j0 && 36 < j0 + K) cd.zeta.d[36 - j0] = T(1);
      if (37 >= j0 && 37 < j0 + K) cd.q0.d[37 - j0] = T(1);
      D v[36];
      for (int j = 0; j < 36; ++j) {
        v[j] = D(in[j]);
        if (j >= j0 && j < j0 + K) v[j].d[j - j0] = T(1);
      }
      D q0[5], p0, dq[3][5], lapq[5], dp[3], lapp, hp[6];
      for (int k = 0; k < 5; ++k) q0[k] = v[k];
      p0 = v[5];
      for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 5; ++k) dq[a][k] = v[6 + 5 * a + k];
      for (int k = 0; k < 5; ++k) lapq[k] = v[21 + k];
      for (int a = 0; a < 3; ++a) dp[a] = v[26 + a];
      lapp = v[29];
      for (int k = 0; k < 6; ++k) hp[k] = v[30 + k];
      D H[5], mu, sig[9];
      local_fields<D>(cd, q0, p0, dq, lapq, dp, lapp, hp, H, mu, sig);
      for (int k = 0; k < K && j0 + k < 38; ++k) {
        T acc2 = T(0);
        for (int c = 0; c < 5; ++c) acc2 += lo[c] * H[c].d[k];
        acc2 += lo[5] * mu.d[k];
        for (int c = 0; c < 9; ++c) acc2 += lo[6 + c] * sig[c].d[k];
        const int j = j0 + k;
        if (j < 36) A.Bf[j * N + s] = acc2;
        else if (j == 36) pz = (double)acc2;
        else pq = (double)acc2;
      }
    }
  }
  // per-block FP64 sums of the parameter gradients (fixed order: deterministic)
  __shared__ double sh[2][kAdjBlock / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    pz += __shfl_down_sync(0xffffffffu, pz, o);
    pq += __shfl_down_sync(0xffffffffu, pq, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sh[0][wid] = pz; sh[1][wid] = pq; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a0 = 0.0, a1 = 0.0;
    for (int w = 0; w < kAdjBlock / 32; ++w) { a0 += sh[0][w]; a1 += sh[1][w]; }
    A.pgrad[2 * blockIdx.x] = a0;
    A.pgrad[2 * blockIdx.x + 1] = a1;
  }
}

// ---------------------------------------------------------------- RK4
// Transposes of gather_fields, added to the partial cotangents of Q and psi:
//   d_a f(x) = sum_i 3 w_i c_ia f(x + c_i),  lap f(x) = sum_i lw_i f(x + c_i) - 4 f(x),
//   hess_aa f(x) = f(x + e_a) + f(x - e_a) - 2 f(x),
//   hess_ab f(x) = 1/4 sum_{edges in the ab plane} c_a c_b f(x + c).
template <typename T>
__global__ void __launch_bounds__(kAdjBlock) k_adj_gather(AdjDesc<T> A) {
  const InstDesc<T>& I = A.I;
  const long long N = I.N;
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  const int nx = I.nx, ny = I.ny, nz = I.nz;
  const int x = (int)(s % nx);
  const long long t = s / nx;
  const int y = (int)(t % ny), z = (int)(t / ny);
  const Nbr nb = make_nbr(x, y, z, nx, ny, nz);
  const T* __restrict__ b = A.Bf;
  T lq[5], lp;
  for (int k = 0; k < 5; ++k) lq[k] = b[k * N + s] - T(4) * b[(21 + k) * N + s];
  lp = b[5 * N + s] - T(4) * b[29 * N + s] - T(2) * (b[30 * N + s] + b[31 * N + s] + b[32 * N + s]);
#pragma unroll
  for (int i = 1; i < 19; ++i) {
    const int cx = lat_c(i, 0), cy = lat_c(i, 1), cz = lat_c(i, 2);
    const long long m = nb.off(-cx, -cy, -cz);  // x = y - c_i reads f(y) through c_i
    const bool face = lat_c2(i) == 1;
    const T gw = face ? T(1.0 / 6.0) : T(1.0 / 12.0);
    const T lw = face ? T(1.0 / 3.0) : T(1.0 / 6.0);
    const int cc[3] = {cx, cy, cz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (cc[a] == 0) continue;
      const T w = cc[a] > 0 ? gw : -gw;
#pragma unroll
      for (int k = 0; k < 5; ++k) lq[k] += w * b[(6 + 5 * a + k) * N + m];
      lp += w * b[(26 + a) * N + m];
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) lq[k] += lw * b[(21 + k) * N + m];
    lp += lw * b[29 * N + m];
    if (face) {
      const int a = cx ? 0 : (cy ? 1 : 2);
      lp += b[(30 + a) * N + m];
    } else {
      const T sgn = T(0.25) * T(cx * cy + cx * cz + cy * cz);
      const int k = (cz == 0) ? 3 : (cy == 0 ? 4 : 5);
      lp += sgn * b[(30 + k) * N + m];
    }
  }
  for (int k = 0; k < 5; ++k) A.oq[k * N + s] += lq[k];
  A.op[s] += lp;
}

// ---------------------------------------------------------------- objective seed
// J = |X(T) - X(0)|^2 / 2 with X_a = (L_a / 2 pi) atan2(S_a, C_a), S_a = sum phi_c sin,
// C_a = sum phi_c cos, phi_c = (1 + psi)/2.  dJ/dpsi(x) = sum_a dX_a coef_a
// (C_a sin th_a(x) - S_a cos th_a(x)) / 2, coef_a = (L_a / 2 pi) / (C_a^2 + S_a^2).
template <typename T>
__global__ void k_adj_seed(InstDesc<T> I, double dX0, double dX1, double dX2, double k0s, double k0c, double k1s,
                           double k1c, double k2s, double k2c, T* lp) {
  const long long N = I.N;
  const double two_pi = 6.283185307179586476925286766559;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N; s += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(s % I.nx);
    const long long t = s / I.nx;
    const int y = (int)(t % I.ny), z = (int)(t / I.ny);
    double sx, cx, sy, cy, sz, cz;
    sincos(two_pi * x / I.nx, &sx, &cx);
    sincos(two_pi * y / I.ny, &sy, &cy);
    sincos(two_pi * z / I.nz, &sz, &cz);
    const double v = 0.5 * (dX0 * (k0s * sx - k0c * cx) + dX1 * (k1s * sy - k1c * cy) + dX2 * (k2s * sz - k2c * cz));
    lp[s] = (T)v;
  }
}

// Cotangent of a stored state, written in the lbcad_get_fields layout: populations as the
// pre-collision f_i(x) = g*_i(x - c_i) (so lam f_i(x) = lam g*_i(x - c_i)), then U, Q, PSI.
template <typename T>
__global__ void k_adj_export(InstDesc<T> I, const T* __restrict__ lg, const T* __restrict__ lq,
                             const T* __restrict__ lp, const T* __restrict__ lu, long long oG, long long oU,
                             long long oQ, long long oP, double* __restrict__ dst) {
  const long long N = I.N;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N; s += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(s % I.nx);
    const long long t = s / I.nx;
    const int y = (int)(t % I.ny), z = (int)(t / I.ny);
    if (oG >= 0) {
      const Nbr nb = make_nbr(x, y, z, I.nx, I.ny, I.nz);
#pragma unroll
      for (int i = 0; i < 19; ++i)
        dst[oG + i * N + s] = (double)lg[i * N + nb.off(-lat_c(i, 0), -lat_c(i, 1), -lat_c(i, 2))];
    }
    if (oU >= 0)
      for (int a = 0; a < 3; ++a) dst[oU + a * N + s] = (double)lu[a * N + s];
    if (oQ >= 0)
      for (int k = 0; k < 5; ++k) dst[oQ + k * N + s] = (double)lq[k * N + s];
    if (oP >= 0) dst[oP + s] = (double)lp[s];
  }
}

// ---------------------------------------------------------------- launchers
template <typename T, bool SHIFT>
cudaError_t LaunchAdj<T, SHIFT>::export_fields(const InstDesc<T>& I, const T* lam, uint32_t mask, double* dst,
                                               cudaStream_t s) {
  const long long N = I.N;
  long long o = 0, oG = -1, oU = -1, oQ = -1, oP = -1;
  if (mask & 1u) { oG = o; o += 19 * N; }
  if (mask & 4u) { oU = o; o += 3 * N; }
  if (mask & 8u) { oQ = o; o += 5 * N; }
  if (mask & 16u) { oP = o; o += N; }
  k_adj_export<T><<<grid_for(N, 256), 256, 0, s>>>(I, lam, lam + 19 * N, lam + 24 * N, lam + 25 * N, oG, oU, oQ, oP,
                                                     dst);
  return cudaGetLastError();
}
template <typename T, bool SHIFT>
cudaError_t LaunchAdj<T, SHIFT>::reverse_step(const AdjDescHost<T>& h, cudaStream_t s) {
  AdjDesc<T> A;
  A.I = h.I;
  A.lg = h.lg; A.lq = h.lq; A.lp = h.lp; A.lu = h.lu;
  A.A = h.A; A.Bf = h.Bf; A.ls = h.ls;
  A.og = h.og; A.oq = h.oq; A.op = h.op; A.ou = h.ou;
  A.pgrad = h.pgrad;
  const unsigned nb = (unsigned)((h.I.N + kAdjBlock - 1) / kAdjBlock);
  constexpr int K = sizeof(T) == 4 ? 8 : 4;
  k_adj_update<T, SHIFT><<<nb, kAdjBlock, 0, s>>>(A);
  k_adj_spread<T><<<nb, kAdjBlock, 0, s>>>(A);
  k_adj_fields<T, K><<<nb, kAdjBlock, 0, s>>>(A);
  k_adj_gather<T><<<nb, kAdjBlock, 0, s>>>(A);
  return cudaGetLastError();
}

template <typename T, bool SHIFT>
int LaunchAdj<T, SHIFT>::blocks(long long N) {
  return (int)((N + kAdjBlock - 1) / kAdjBlock);
}

template <typename T, bool SHIFT>
cudaError_t LaunchAdj<T, SHIFT>::seed(const InstDesc<T>& I, const double dX[3], const double ks[3],
                                      const double kc[3], T* lp, cudaStream_t s) {
  k_adj_seed<T><<<grid_for(I.N, 256), 256, 0, s>>>(I, dX[0], dX[1], dX[2], ks[0], kc[0], ks[1], kc[1], ks[2], kc[2], lp);
  return cudaGetLastError();
}

}  // namespace lbcad
