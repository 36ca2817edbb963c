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
//                      to its 36 inputs (Q, psi and their stencils) and to zeta and q0, by a
//                      hand-written reverse sweep (local_fields_vjp)
//   RK4 k_adj_gather : transposes of the Q/psi stencils (gradient, Laplacian, Hessian)
// The per-site reverse sweeps recompute the forward intermediates of the site and take
// every branch (upwind sides) as the forward takes it.  Stencil transposes use the negated offsets on the
// periodic lattice, so no site is written by two threads.
#pragma once

#include "lbcad_kernels.cuh"

namespace lbcad {

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

// ---------------------------------------------------------------- reverse mode of local_fields
// Vector-Jacobian product of local_fields at one site by a hand-written reverse sweep: in =
// the 36 inputs (q0 0-4, psi 5, dq 6-20 as 6 + 5a + k, lapq 21-25, dp 26-28, lapp 29,
// hp 30-35), lo = the cotangents of its outputs (H 0-4, mu 5, sigma 6-14), out = the
// cotangents of the 36 inputs; lzeta and lq0 receive the derivatives with respect to the
// parameters zeta and q0.  Full 3x3 cotangents of Q and dQ_a are accumulated entry by entry
// as the forward reads them and folded onto the five stored components at the end.
template <typename T>
__device__ __forceinline__ void local_fields_vjp(const Coef<T>& c, const T in[36], const T lo[15], T out[36],
                                                 T& lzeta, T& lq0) {
  // ---- forward intermediates
  const T* q = in;
  const T psi = in[5];
  T Q[3][3];
  full3(q, Q);
  T dQ[3][3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) full3(in + 6 + 5 * a, dQ[a]);
  const T* dp = in + 26;
  const T* hp = in + 30;
  const T chi = c.chi0 + c.chis * (T(1) + psi);
  T QQ[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      QQ[i][j] = Q[i][0] * Q[0][j] + Q[i][1] * Q[1][j] + Q[i][2] * Q[2][j];
      QQ[j][i] = QQ[i][j];
    }
  const T trQ2 = QQ[0][0] + QQ[1][1] + QQ[2][2];
  const T trQ3 = QQ[0][0] * Q[0][0] + QQ[1][1] * Q[1][1] + QQ[2][2] * Q[2][2] +
                 T(2) * (QQ[0][1] * Q[0][1] + QQ[0][2] * Q[0][2] + QQ[1][2] * Q[1][2]);
  T C[3][3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    C[0][b] = dQ[1][2][b] - dQ[2][1][b];
    C[1][b] = dQ[2][0][b] - dQ[0][2][b];
    C[2][b] = dQ[0][1][b] - dQ[1][0][b];
  }
  T CC[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) CC[i][j] = C[i][j] + C[j][i];
  const T g2 = dp[0] * dp[0] + dp[1] * dp[1] + dp[2] * dp[2];
  const T Ac = c.A0 * chi;
  const T Kq = T(2) * c.K * c.q0;
  const T lin = -c.A0 * (T(1) - chi / T(3)) - Ac * trQ2 - Kq * T(2) * c.q0;
  const T iso = (Ac * trQ2 - c.W * g2) / T(3);
  const int I5[5] = {0, 0, 0, 1, 1};
  const int J5[5] = {0, 1, 2, 1, 2};
  T H[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int i = I5[k], j = J5[k];
    T h = lin * Q[i][j] + Ac * QQ[i][j] + c.K * in[21 + k] - Kq * CC[i][j] - c.W * dp[i] * dp[j];
    if (i == j) h -= iso;
    H[k] = h;
  }
  T Hf[3][3];
  full3(H, Hf);
  const T Qh = Q[0][0] * hp[0] + Q[1][1] * hp[1] + Q[2][2] * hp[2] +
               T(2) * (Q[0][1] * hp[3] + Q[0][2] * hp[4] + Q[1][2] * hp[5]);
  T divQdp = T(0);
#pragma unroll
  for (int b = 0; b < 3; ++b) divQdp += (dQ[0][0][b] + dQ[1][1][b] + dQ[2][2][b]) * dp[b];
  const T psi2 = psi * psi;
  const T mu = psi * (c.b * psi2 - c.a) - c.kphi * in[29] +
               c.A0 * c.chis * (trQ2 * (T(0.25) * trQ2 - T(1) / T(6)) - trQ3 / T(3)) - T(2) * c.W * (divQdp + Qh);
  T Qdp[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) Qdp[i] = Q[i][0] * dp[0] + Q[i][1] * dp[1] + Q[i][2] * dp[2];
  const T QC = Q[0][0] * C[0][0] + Q[1][1] * C[1][1] + Q[2][2] * C[2][2] + Q[0][1] * CC[0][1] +
               Q[0][2] * CC[0][2] + Q[1][2] * CC[1][2];
  T QH[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) QH[i][j] = Q[i][0] * Hf[0][j] + Q[i][1] * Hf[1][j] + Q[i][2] * Hf[2][j];
  const T phic = T(0.5) * (T(1) + psi);
  const T trQH = QH[0][0] + QH[1][1] + QH[2][2];
  const T cQ = T(2) * c.xi * trQH - c.zeta * phic;
  const T cH = -T(2) * c.xi / T(3);
  const T cP = T(1) - c.xi, cM = -(T(1) + c.xi);
  T wv[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) wv[b] = c.kphi * dp[b] + T(2) * c.W * Qdp[b];
  T v[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int g = (b + 1) % 3, m = (b + 2) % 3;
      v[a][b] = dQ[a][g][0] * Q[0][m] + dQ[a][g][1] * Q[1][m] + dQ[a][g][2] * Q[2][m] -
                (dQ[a][m][0] * Q[0][g] + dQ[a][m][1] * Q[1][g] + dQ[a][m][2] * Q[2][g]);
    }

  // ---- reverse sweep
  T lQ[3][3], ldQ[3][3][3], lHf[3][3], lQH[3][3], lG[3][3], lCC[3][3], lC[3][3], lQQ[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      lQ[i][j] = lHf[i][j] = lQH[i][j] = lG[i][j] = lCC[i][j] = lC[i][j] = lQQ[i][j] = T(0);
#pragma unroll
      for (int a = 0; a < 3; ++a) ldQ[a][i][j] = T(0);
    }
  T ldp[3] = {T(0), T(0), T(0)}, lwv[3] = {T(0), T(0), T(0)}, lQdp[3] = {T(0), T(0), T(0)};
  T lpsi = T(0), lcQ = T(0), lcI = T(0), lKq = T(0), ltrQH = T(0), lP0 = T(0), lphic = T(0);
  lzeta = T(0);
  lq0 = T(0);
  // sigma
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const T L = lo[6 + 3 * a + b];
      lcQ += L * Q[a][b];
      lQ[a][b] += cQ * L;
      lQH[a][b] += cP * L;
      lQH[b][a] += cM * L;
      lHf[a][b] += cH * L;
      lG[a][b] += -c.K * L;
      lKq += -v[a][b] * L;
      const T lv = -Kq * L;
      ldp[a] += -wv[b] * L;
      lwv[b] += -dp[a] * L;
      if (a == b) lcI += L;
      const int g = (b + 1) % 3, m = (b + 2) % 3;
#pragma unroll
      for (int n = 0; n < 3; ++n) {
        ldQ[a][g][n] += lv * Q[n][m];
        lQ[n][m] += lv * dQ[a][g][n];
        ldQ[a][m][n] -= lv * Q[n][g];
        lQ[n][g] -= lv * dQ[a][m][n];
      }
    }
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    ldp[b] += c.kphi * lwv[b];
    lQdp[b] += T(2) * c.W * lwv[b];
  }
  // cQ = 2 xi trQH - zeta phic; cI = (2 xi/3) trQH - P0
  ltrQH += T(2) * c.xi * lcQ + (T(2) * c.xi / T(3)) * lcI;
  lzeta += -phic * lcQ;
  lphic += -c.zeta * lcQ;
  lP0 += -lcI;
  lpsi += T(0.5) * lphic;
#pragma unroll
  for (int i = 0; i < 3; ++i) lQH[i][i] += ltrQH;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        lQ[i][m] += lQH[i][j] * Hf[m][j];
        lHf[m][j] += Q[i][m] * lQH[i][j];
      }
  // P0 = psi mu - fden
  const T lmu = lo[5] + psi * lP0;
  lpsi += mu * lP0;
  const T lf = -lP0;
  // fden
  T lpsi2 = (T(0.5) * c.b * psi2 - T(0.5) * c.a) * lf;
  T lg2 = T(0.5) * c.kphi * lf;
  T lchi = c.A0 * (-(T(0.5) / T(3)) * trQ2 - trQ3 / T(3) + trQ2 * trQ2 / T(4)) * lf;
  T ltrQ2 = c.A0 * (T(0.5) * (T(1) - chi / T(3)) + chi / T(2) * trQ2) * lf + Kq * c.q0 * lf;
  T ltrQ3 = -c.A0 * chi / T(3) * lf;
#pragma unroll
  for (int a = 0; a < 3; ++a) lG[a][a] += T(0.5) * c.K * lf;
  lKq += QC * lf + c.q0 * trQ2 * lf;
  const T lQC = Kq * lf;
  lq0 += Kq * trQ2 * lf;
  const T lanch = c.W * lf;
  // anch = dp . Qdp; Qdp = Q dp
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    ldp[i] += Qdp[i] * lanch;
    lQdp[i] += dp[i] * lanch;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      lQ[i][m] += lQdp[i] * dp[m];
      ldp[m] += Q[i][m] * lQdp[i];
    }
  // QC
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    lQ[i][i] += C[i][i] * lQC;
    lC[i][i] += Q[i][i] * lQC;
  }
  lQ[0][1] += CC[0][1] * lQC;
  lCC[0][1] += Q[0][1] * lQC;
  lQ[0][2] += CC[0][2] * lQC;
  lCC[0][2] += Q[0][2] * lQC;
  lQ[1][2] += CC[1][2] * lQC;
  lCC[1][2] += Q[1][2] * lQC;
  // mu
  lpsi += (c.b * psi2 - c.a) * lmu;
  lpsi2 += psi * c.b * lmu;
  T llapp = -c.kphi * lmu;
  ltrQ2 += c.A0 * c.chis * (T(0.5) * trQ2 - T(1) / T(6)) * lmu;
  ltrQ3 += -c.A0 * c.chis / T(3) * lmu;
  const T ldiv = -T(2) * c.W * lmu, lQh = -T(2) * c.W * lmu;
  // Qh
  T lhp[6];
  lQ[0][0] += hp[0] * lQh;
  lQ[1][1] += hp[1] * lQh;
  lQ[2][2] += hp[2] * lQh;
  lQ[0][1] += T(2) * hp[3] * lQh;
  lQ[0][2] += T(2) * hp[4] * lQh;
  lQ[1][2] += T(2) * hp[5] * lQh;
  lhp[0] = Q[0][0] * lQh;
  lhp[1] = Q[1][1] * lQh;
  lhp[2] = Q[2][2] * lQh;
  lhp[3] = T(2) * Q[0][1] * lQh;
  lhp[4] = T(2) * Q[0][2] * lQh;
  lhp[5] = T(2) * Q[1][2] * lQh;
  // divQdp
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    ldQ[0][0][b] += dp[b] * ldiv;
    ldQ[1][1][b] += dp[b] * ldiv;
    ldQ[2][2][b] += dp[b] * ldiv;
    ldp[b] += (dQ[0][0][b] + dQ[1][1][b] + dQ[2][2][b]) * ldiv;
  }
  lpsi += T(2) * psi * lpsi2;
  // G (symmetric): the computed value s_ab serves G[a][b] and G[b][a]
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = a; b < 3; ++b) {
      const T ls = (a == b) ? lG[a][a] : lG[a][b] + lG[b][a];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
          const T w = (i == j) ? T(1) : T(2);
          ldQ[a][i][j] += w * ls * dQ[b][i][j];
          ldQ[b][i][j] += w * ls * dQ[a][i][j];
        }
    }
  // H (outputs and the uses of Hf)
  T lH[5];
  lH[0] = lo[0] + lHf[0][0] - lHf[2][2];
  lH[1] = lo[1] + lHf[0][1] + lHf[1][0];
  lH[2] = lo[2] + lHf[0][2] + lHf[2][0];
  lH[3] = lo[3] + lHf[1][1] - lHf[2][2];
  lH[4] = lo[4] + lHf[1][2] + lHf[2][1];
  T llin = T(0), lAc = T(0), liso = T(0), llapq[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int i = I5[k], j = J5[k];
    const T L = lH[k];
    llin += Q[i][j] * L;
    lQ[i][j] += lin * L;
    lAc += QQ[i][j] * L;
    lQQ[i][j] += Ac * L;
    llapq[k] = c.K * L;
    lKq += -CC[i][j] * L;
    lCC[i][j] += -Kq * L;
    ldp[i] += -c.W * dp[j] * L;
    ldp[j] += -c.W * dp[i] * L;
    if (i == j) liso += -L;
  }
  // iso, lin, Kq, Ac, g2
  lAc += trQ2 / T(3) * liso;
  ltrQ2 += Ac / T(3) * liso;
  lg2 += -c.W / T(3) * liso;
  lchi += (c.A0 / T(3)) * llin;
  lAc += -trQ2 * llin;
  ltrQ2 += -Ac * llin;
  lKq += -T(2) * c.q0 * llin;
  lq0 += -T(2) * Kq * llin;
  lq0 += T(2) * c.K * lKq;
  lchi += c.A0 * lAc;
#pragma unroll
  for (int b = 0; b < 3; ++b) ldp[b] += T(2) * dp[b] * lg2;
  // CC (symmetric value per unordered pair) and C
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      if (i == j) {
        lC[i][i] += T(2) * lCC[i][i];
      } else {
        const T l = lCC[i][j] + lCC[j][i];
        lC[i][j] += l;
        lC[j][i] += l;
      }
    }
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    ldQ[1][2][b] += lC[0][b];
    ldQ[2][1][b] -= lC[0][b];
    ldQ[2][0][b] += lC[1][b];
    ldQ[0][2][b] -= lC[1][b];
    ldQ[0][1][b] += lC[2][b];
    ldQ[1][0][b] -= lC[2][b];
  }
  // trQ3, trQ2, QQ
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    lQQ[i][i] += Q[i][i] * ltrQ3 + ltrQ2;
    lQ[i][i] += QQ[i][i] * ltrQ3;
  }
  lQQ[0][1] += T(2) * Q[0][1] * ltrQ3;
  lQ[0][1] += T(2) * QQ[0][1] * ltrQ3;
  lQQ[0][2] += T(2) * Q[0][2] * ltrQ3;
  lQ[0][2] += T(2) * QQ[0][2] * ltrQ3;
  lQQ[1][2] += T(2) * Q[1][2] * ltrQ3;
  lQ[1][2] += T(2) * QQ[1][2] * ltrQ3;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const T l = (i == j) ? lQQ[i][i] : lQQ[i][j] + lQQ[j][i];
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        lQ[i][m] += l * Q[m][j];
        lQ[m][j] += l * Q[i][m];
      }
    }
  // chi = chi0 + chis (1 + psi)
  lpsi += c.chis * lchi;
  // fold the full-matrix cotangents onto the stored components (full3 transposed)
  out[0] = lQ[0][0] - lQ[2][2];
  out[1] = lQ[0][1] + lQ[1][0];
  out[2] = lQ[0][2] + lQ[2][0];
  out[3] = lQ[1][1] - lQ[2][2];
  out[4] = lQ[1][2] + lQ[2][1];
  out[5] = lpsi;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    out[6 + 5 * a + 0] = ldQ[a][0][0] - ldQ[a][2][2];
    out[6 + 5 * a + 1] = ldQ[a][0][1] + ldQ[a][1][0];
    out[6 + 5 * a + 2] = ldQ[a][0][2] + ldQ[a][2][0];
    out[6 + 5 * a + 3] = ldQ[a][1][1] - ldQ[a][2][2];
    out[6 + 5 * a + 4] = ldQ[a][1][2] + ldQ[a][2][1];
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) out[21 + k] = llapq[k];
#pragma unroll
  for (int b = 0; b < 3; ++b) out[26 + b] = ldp[b];
  out[29] = llapp;
#pragma unroll
  for (int k = 0; k < 6; ++k) out[30 + k] = lhp[k];
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
template <typename T>
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
    T ci[36], lz, lq;
    local_fields_vjp<T>(I.c, in, lo, ci, lz, lq);
    for (int j = 0; j < 36; ++j) A.Bf[j * N + s] = ci[j];
    pz = (double)lz;
    pq = (double)lq;
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
  k_adj_update<T, SHIFT><<<nb, kAdjBlock, 0, s>>>(A);
  k_adj_spread<T><<<nb, kAdjBlock, 0, s>>>(A);
  k_adj_fields<T><<<nb, kAdjBlock, 0, s>>>(A);
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
