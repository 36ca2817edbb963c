// lbcad_kernels.cuh -- CUDA kernels of the hybrid LB step, templated on the compute
// type T (float or double) and on SHIFT (populations stored as f_i - w_i rho0).
//
// One step (Sec. 3 of Carenza, Gonnella & Negro) runs as two per-site kernels:
//   k_fields : isotropic D3Q19 stencils of Q and psi -> molecular field H (Eq. 2, 5),
//              chemical potential mu (Eq. 1, 5) and total stress sigma (Eq. 3, 4)
//              into scratch;
//   k_update : F = div sigma, BGK + Guo collision of the pulled populations (Eqs. 6-8),
//              Beris-Edwards update of Q with upwind advection and co-rotation (Eq. 2),
//              Cahn-Hilliard update of psi in upwind flux form (Eq. 1).
// Layout: every field is [component][z][y][x] (x fastest) per instance; neighbour reads
// are coalesced along x and served by L1/L2.
#pragma once

#include "lbcad_internal.h"

namespace lbcad {

template <typename T>
__device__ __forceinline__ T ld(const T* p) {
  return __ldg(p);
}

template <typename T>
__device__ __forceinline__ int find_inst(const InstDesc<T>* __restrict__ D, int n, long long b) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (D[mid].blk0 <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Periodic neighbour offsets of one site: off(dx, dy, dz) for dx, dy, dz in {-1, 0, 1}.
struct Nbr {
  int xo[3];
  int yo[3];
  long long zo[3];
  __device__ __forceinline__ long long off(int dx, int dy, int dz) const {
    return (long long)xo[dx + 1] + yo[dy + 1] + zo[dz + 1];
  }
};

__device__ __forceinline__ Nbr make_nbr(int x, int y, int z, int nx, int ny, int nz) {
  Nbr n;
  n.xo[0] = x ? x - 1 : nx - 1;
  n.xo[1] = x;
  n.xo[2] = (x + 1 < nx) ? x + 1 : 0;
  n.yo[0] = (y ? y - 1 : ny - 1) * nx;
  n.yo[1] = y * nx;
  n.yo[2] = ((y + 1 < ny) ? y + 1 : 0) * nx;
  const long long pl = (long long)nx * ny;
  n.zo[0] = (z ? z - 1 : nz - 1) * pl;
  n.zo[1] = z * pl;
  n.zo[2] = ((z + 1 < nz) ? z + 1 : 0) * pl;
  return n;
}

// Full symmetric traceless tensor from the five stored components xx, xy, xz, yy, yz.
template <typename T>
__device__ __forceinline__ void full3(const T q[5], T Q[3][3]) {
  Q[0][0] = q[0]; Q[0][1] = q[1]; Q[0][2] = q[2];
  Q[1][0] = q[1]; Q[1][1] = q[3]; Q[1][2] = q[4];
  Q[2][0] = q[2]; Q[2][1] = q[4]; Q[2][2] = -q[0] - q[3];
}

// H (5), mu and the total stress sigma (9, row-major a*3+b) at one site from Q, psi and
// their stencils: dq[a][k] = d_a of stored component k, lapq[k], dp[a] = d_a psi,
// lapp, hp = Hessian of psi (xx, yy, zz, xy, xz, yz).
template <typename T>
__device__ __forceinline__ void local_fields(const Coef<T>& c, const T q[5], T psi, const T dq[3][5],
                                             const T lapq[5], const T dp[3], T lapp, const T hp[6], T H[5],
                                             T& mu, T sig[9]) {
  T Q[3][3];
  full3(q, Q);
  T dQ[3][3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) full3(dq[a], dQ[a]);
  const T chi = c.chi0 + c.chis * (T(1) + psi);
  T QQ[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) QQ[i][j] = Q[i][0] * Q[0][j] + Q[i][1] * Q[1][j] + Q[i][2] * Q[2][j];
  const T trQ2 = QQ[0][0] + QQ[1][1] + QQ[2][2];
  T trQ3 = T(0);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) trQ3 += QQ[i][j] * Q[i][j];
  // curl: C_ab = eps_amn d_m Q_nb
  T C[3][3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    C[0][b] = dQ[1][2][b] - dQ[2][1][b];
    C[1][b] = dQ[2][0][b] - dQ[0][2][b];
    C[2][b] = dQ[0][1][b] - dQ[1][0][b];
  }
  const T g2 = dp[0] * dp[0] + dp[1] * dp[1] + dp[2] * dp[2];
  const T lin = -c.A0 * (T(1) - chi / T(3)) - c.A0 * chi * trQ2 - T(4) * c.K * c.q0 * c.q0;
  const T Ac = c.A0 * chi;
  const T Kq = T(2) * c.K * c.q0;
  // H = -dF/dQ, symmetric traceless by construction (C + C^T is traceless for symmetric Q)
  const int I5[5] = {0, 0, 0, 1, 1};
  const int J5[5] = {0, 1, 2, 1, 2};
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int i = I5[k], j = J5[k];
    const T dij = (i == j) ? T(1) : T(0);
    H[k] = lin * Q[i][j] + Ac * (QQ[i][j] - dij * trQ2 / T(3)) + c.K * lapq[k] - Kq * (C[i][j] + C[j][i]) -
           c.W * (dp[i] * dp[j] - dij * g2 / T(3));
  }
  T Hf[3][3];
  full3(H, Hf);

  // mu = dF/dpsi
  T Qh = Q[0][0] * hp[0] + Q[1][1] * hp[1] + Q[2][2] * hp[2] +
         T(2) * (Q[0][1] * hp[3] + Q[0][2] * hp[4] + Q[1][2] * hp[5]);
  T divQdp = T(0);
#pragma unroll
  for (int b = 0; b < 3; ++b) divQdp += (dQ[0][0][b] + dQ[1][1][b] + dQ[2][2][b]) * dp[b];
  mu = -c.a * psi + c.b * psi * psi * psi - c.kphi * lapp +
       c.A0 * c.chis * (-trQ2 / T(6) - trQ3 / T(3) + trQ2 * trQ2 / T(4)) - T(2) * c.W * (divQdp + Qh);

  // Gram matrix of the Q derivatives and the free-energy density
  T G[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = a; b < 3; ++b) {
      T s = T(0);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) s += dQ[a][i][j] * dQ[b][i][j];
      G[a][b] = s;
      G[b][a] = s;
    }
  T QC = T(0);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) QC += Q[i][j] * C[i][j];
  T Qdp[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) Qdp[i] = Q[i][0] * dp[0] + Q[i][1] * dp[1] + Q[i][2] * dp[2];
  const T anch = dp[0] * Qdp[0] + dp[1] * Qdp[1] + dp[2] * Qdp[2];
  const T psi2 = psi * psi;
  const T fden = -T(0.5) * c.a * psi2 + T(0.25) * c.b * psi2 * psi2 + T(0.5) * c.kphi * g2 +
                 c.A0 * (T(0.5) * (T(1) - chi / T(3)) * trQ2 - chi / T(3) * trQ3 + chi / T(4) * trQ2 * trQ2) +
                 T(0.5) * c.K * (G[0][0] + G[1][1] + G[2][2]) + Kq * QC + T(2) * c.K * c.q0 * c.q0 * trQ2 +
                 c.W * anch;
  const T P0 = psi * mu - fden;

  // reactive parts: QH, HQ, tr(QH)
  T QH[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) QH[i][j] = Q[i][0] * Hf[0][j] + Q[i][1] * Hf[1][j] + Q[i][2] * Hf[2][j];
  const T trQH = QH[0][0] + QH[1][1] + QH[2][2];
  const T phic = T(0.5) * (T(1) + psi);

#pragma unroll
  for (int a = 0; a < 3; ++a) {
    // axial vector of the antisymmetric part of dQ_a . Q: v_b = eps_bgm (dQ_a Q)_gm
    T A[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) A[i][j] = dQ[a][i][0] * Q[0][j] + dQ[a][i][1] * Q[1][j] + dQ[a][i][2] * Q[2][j];
    const T v[3] = {A[1][2] - A[2][1], A[2][0] - A[0][2], A[0][1] - A[1][0]};
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const T dab = (a == b) ? T(1) : T(0);
      // QH^T = HQ for symmetric Q, H: (HQ)_ab = QH_ba
      const T HQab = QH[b][a];
      T s = -P0 * dab - c.K * G[a][b] - Kq * v[b] - dp[a] * (c.kphi * dp[b] + T(2) * c.W * Qdp[b]);
      s += -c.xi * (HQab + QH[a][b]) - (T(2) * c.xi / T(3)) * Hf[a][b] +
           T(2) * c.xi * trQH * (Q[a][b] + dab / T(3)) + (QH[a][b] - HQab);
      s += -c.zeta * phic * Q[a][b];
      sig[3 * a + b] = s;
    }
  }
}

// ---------------------------------------------------------------- k_fields
template <typename T>
__global__ void __launch_bounds__(kStepBlock) k_fields(const InstDesc<T>* __restrict__ D, int ninst) {
  const int ii = find_inst(D, ninst, (long long)blockIdx.x);
  const InstDesc<T>& I = D[ii];
  const long long N = I.N;
  const long long s = ((long long)blockIdx.x - I.blk0) * blockDim.x + threadIdx.x;
  if (s >= N) return;
  const int nx = I.nx, ny = I.ny, nz = I.nz;
  const int x = (int)(s % nx);
  const long long t = s / nx;
  const int y = (int)(t % ny);
  const int z = (int)(t / ny);
  const Nbr nb = make_nbr(x, y, z, nx, ny, nz);
  const T* __restrict__ q = I.q_in;
  const T* __restrict__ ps = I.psi_in;

  T q0[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) q0[k] = ld(q + k * N + s);
  const T p0 = ld(ps + s);
  T dq[3][5], lapq[5], dp[3], hp[6];
  T lapp = T(0);
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    lapq[k] = T(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) dq[a][k] = T(0);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) dp[a] = T(0);
#pragma unroll
  for (int k = 0; k < 6; ++k) hp[k] = T(0);

#pragma unroll
  for (int i = 1; i < 19; ++i) {
    const int cx = lat_c(i, 0), cy = lat_c(i, 1), cz = lat_c(i, 2);
    const long long n = nb.off(cx, cy, cz);
    // differences to the centre value: Sum_i w_i c_i = 0 makes every stencil below a
    // sum of differences, which keeps FP32 Laplacians free of cancellation
    T qn[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) qn[k] = ld(q + k * N + n) - q0[k];
    const T pn = ld(ps + n) - p0;
    const bool face = lat_c2(i) == 1;
    const T gw = face ? T(1.0 / 6.0) : T(1.0 / 12.0);
    const T lw = face ? T(1.0 / 3.0) : T(1.0 / 6.0);
    const int cc[3] = {cx, cy, cz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (cc[a] == 0) continue;
      const T wa = cc[a] > 0 ? gw : -gw;
#pragma unroll
      for (int k = 0; k < 5; ++k) dq[a][k] += wa * qn[k];
      dp[a] += wa * pn;
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) lapq[k] += lw * qn[k];
    lapp += lw * pn;
    if (face) {
      const int a = cx ? 0 : (cy ? 1 : 2);
      hp[a] += pn;
    } else {
      const T sgn = T(0.25) * T(cx * cy + cx * cz + cy * cz);  // c_a c_b of the two non-zero axes
      const int k = (cz == 0) ? 3 : (cy == 0 ? 4 : 5);          // xy, xz, yz
      hp[k] += sgn * pn;
    }
  }

  T H[5], sig[9], mu;
  local_fields<T>(I.c, q0, p0, dq, lapq, dp, lapp, hp, H, mu, sig);
#pragma unroll
  for (int k = 0; k < 5; ++k) I.H[k * N + s] = H[k];
  I.mu[s] = mu;
#pragma unroll
  for (int k = 0; k < 9; ++k) I.sig[k * N + s] = sig[k];
}

// ---------------------------------------------------------------- k_update
template <typename T, bool SHIFT>
__global__ void __launch_bounds__(kStepBlock) k_update(const InstDesc<T>* __restrict__ D, int ninst) {
  const int ii = find_inst(D, ninst, (long long)blockIdx.x);
  const InstDesc<T>& I = D[ii];
  const long long N = I.N;
  const long long s = ((long long)blockIdx.x - I.blk0) * blockDim.x + threadIdx.x;
  if (s >= N) return;
  const int nx = I.nx, ny = I.ny, nz = I.nz;
  const int x = (int)(s % nx);
  const long long t = s / nx;
  const int y = (int)(t % ny);
  const int z = (int)(t / ny);
  const Nbr nb = make_nbr(x, y, z, nx, ny, nz);
  const Coef<T> c = I.c;
  const T* __restrict__ sg = I.sig;
  const T* __restrict__ mu = I.mu;
  const T* __restrict__ ui = I.u_in;
  const T* __restrict__ q = I.q_in;
  const T* __restrict__ ps = I.psi_in;

  T s0[9], u0[3];
#pragma unroll
  for (int k = 0; k < 9; ++k) s0[k] = ld(sg + k * N + s);
#pragma unroll
  for (int a = 0; a < 3; ++a) u0[a] = ld(ui + a * N + s);
  const T mu0 = ld(mu + s);
  T F[3] = {T(0), T(0), T(0)};
  T Wg[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) Wg[a][b] = T(0);
  T lapmu = T(0);
  T qf[6][5], pf[6], uf[6];
#pragma unroll
  for (int i = 1; i < 19; ++i) {
    const int cx = lat_c(i, 0), cy = lat_c(i, 1), cz = lat_c(i, 2);
    const long long n = nb.off(cx, cy, cz);
    const bool face = lat_c2(i) == 1;
    const T gw = face ? T(1.0 / 6.0) : T(1.0 / 12.0);
    const T lw = face ? T(1.0 / 3.0) : T(1.0 / 6.0);
    lapmu += lw * (ld(mu + n) - mu0);
    T un[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) un[a] = ld(ui + a * N + n);
    const int cc[3] = {cx, cy, cz};
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (cc[b] == 0) continue;
      const T wb = cc[b] > 0 ? gw : -gw;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        F[a] += wb * (ld(sg + (3 * a + b) * N + n) - s0[3 * a + b]);
        Wg[a][b] += wb * (un[a] - u0[a]);
      }
    }
    if (face) {
      const int a = cx ? 0 : (cy ? 1 : 2);
#pragma unroll
      for (int k = 0; k < 5; ++k) qf[i - 1][k] = ld(q + k * N + n);
      pf[i - 1] = ld(ps + n);
      uf[i - 1] = un[a];
    }
  }

  // ---- Beris-Edwards update of Q (Eq. 2) with u of the previous step
  T q0[5], Hs[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    q0[k] = ld(q + k * N + s);
    Hs[k] = I.H[k * N + s];
  }
  const T p0 = ld(ps + s);
  T adv[5] = {T(0), T(0), T(0), T(0), T(0)};
  T divJ = T(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int ip = 2 * a, im = 2 * a + 1;  // face slots of +e_a, -e_a
    const T up = u0[a] > T(0) ? u0[a] : T(0);
    const T um = u0[a] < T(0) ? u0[a] : T(0);
#pragma unroll
    for (int k = 0; k < 5; ++k) adv[k] += up * (q0[k] - qf[im][k]) + um * (qf[ip][k] - q0[k]);
    const T ubp = T(0.5) * (u0[a] + uf[ip]);
    const T Jp = ubp * (ubp > T(0) ? p0 : pf[ip]);
    const T ubm = T(0.5) * (uf[im] + u0[a]);
    const T Jm = ubm * (ubm > T(0) ? pf[im] : p0);
    divJ += Jp - Jm;
  }
  T Q[3][3];
  full3(q0, Q);
  T Dm[3][3], Om[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Dm[i][j] = T(0.5) * (Wg[i][j] + Wg[j][i]);
      Om[i][j] = T(0.5) * (Wg[i][j] - Wg[j][i]);
    }
  T trQW = T(0);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) trQW += Q[i][j] * Wg[j][i];
  const T trD = Dm[0][0] + Dm[1][1] + Dm[2][2];
  const int I5[5] = {0, 0, 0, 1, 1};
  const int J5[5] = {0, 1, 2, 1, 2};
  T qn[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int i = I5[k], j = J5[k];
    const T dij = (i == j) ? T(1) : T(0);
    T DQ = T(0), QD = T(0), OQ = T(0), QO = T(0);
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      DQ += Dm[i][m] * Q[m][j];
      QD += Q[i][m] * Dm[m][j];
      OQ += Om[i][m] * Q[m][j];
      QO += Q[i][m] * Om[m][j];
    }
    // S projected to its traceless part (its trace is 2 xi tr(D)/3)
    const T S = c.xi * (DQ + QD) + (T(2) * c.xi / T(3)) * Dm[i][j] + (OQ - QO) -
                T(2) * c.xi * trQW * (Q[i][j] + dij / T(3)) - dij * (T(2) * c.xi / T(9)) * trD;
    qn[k] = q0[k] - adv[k] + S + c.gammaQ * Hs[k];
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) I.q_out[k * N + s] = qn[k];
  // ---- Cahn-Hilliard update of psi (Eq. 1)
  I.psi_out[s] = p0 - divJ + c.M * lapmu;

  // ---- LB: pull, BGK + Guo collision (Eqs. 6-8), write post-collision at s
  T g[19];
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    const long long src = nb.off(-lat_c(i, 0), -lat_c(i, 1), -lat_c(i, 2));
    g[i] = ld(I.g_in + i * N + src);
  }
  T m0 = T(0), j[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    m0 += g[i];
    if (lat_c(i, 0)) j[0] += lat_c(i, 0) > 0 ? g[i] : -g[i];
    if (lat_c(i, 1)) j[1] += lat_c(i, 1) > 0 ? g[i] : -g[i];
    if (lat_c(i, 2)) j[2] += lat_c(i, 2) > 0 ? g[i] : -g[i];
  }
  const T rho = SHIFT ? (c.rho0 + m0) : m0;
  const T rinv = T(1) / rho;
  T u[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) u[a] = (j[a] + T(0.5) * F[a]) * rinv;
  const T u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const T uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    const T w = T(lat_w(i));
    const T cu = T(lat_c(i, 0)) * u[0] + T(lat_c(i, 1)) * u[1] + T(lat_c(i, 2)) * u[2];
    const T cF = T(lat_c(i, 0)) * F[0] + T(lat_c(i, 1)) * F[1] + T(lat_c(i, 2)) * F[2];
    const T poly = T(3) * cu + T(4.5) * cu * cu - T(1.5) * u2;
    const T geq = SHIFT ? w * (m0 + rho * poly) : w * rho * (T(1) + poly);
    const T Fi = c.guo * w * (T(3) * (cF - uF) + T(9) * cu * cF);
    I.g_out[i * N + s] = g[i] - (g[i] - geq) * c.tau_inv + Fi;
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) I.u_out[a * N + s] = u[a];
}

// ---------------------------------------------------------------- field exchange
// dst components, in mask order: G(19) RHO(1) U(3) Q(5) PSI(1); offsets given per group
// (-1 = not selected).
template <typename T, bool SHIFT>
__global__ void k_get_fields(InstDesc<T> I, long long oG, long long oR, long long oU, long long oQ,
                             long long oP, double* __restrict__ dst) {
  const long long N = I.N;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N; s += (long long)gridDim.x * blockDim.x) {
    const int nx = I.nx, ny = I.ny, nz = I.nz;
    const int x = (int)(s % nx);
    const long long t = s / nx;
    const int y = (int)(t % ny);
    const int z = (int)(t / ny);
    if (oG >= 0 || oR >= 0) {
      const Nbr nb = make_nbr(x, y, z, nx, ny, nz);
      double rho = 0.0;
#pragma unroll
      for (int i = 0; i < 19; ++i) {
        const long long src = nb.off(-lat_c(i, 0), -lat_c(i, 1), -lat_c(i, 2));
        double fi = (double)I.g_in[i * N + src];
        if (SHIFT) fi += lat_w(i) * (double)I.c.rho0;
        rho += fi;
        if (oG >= 0) dst[oG + i * N + s] = fi;
      }
      if (oR >= 0) dst[oR + s] = rho;
    }
    if (oU >= 0)
      for (int a = 0; a < 3; ++a) dst[oU + a * N + s] = (double)I.u_in[a * N + s];
    if (oQ >= 0)
      for (int k = 0; k < 5; ++k) dst[oQ + k * N + s] = (double)I.q_in[k * N + s];
    if (oP >= 0) dst[oP + s] = (double)I.psi_in[s];
  }
}

// Writes pre-collision populations f_i(x) as the stored post-collision array of the
// previous step: stored_i(x - c_i) = f_i(x) (- w_i rho0 when SHIFT).
template <typename T, bool SHIFT>
__global__ void k_set_fields(InstDesc<T> I, long long oG, long long oU, long long oQ, long long oP,
                             const double* __restrict__ src, T* g_t, T* q_t, T* p_t, T* u_t) {
  const long long N = I.N;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N; s += (long long)gridDim.x * blockDim.x) {
    const int nx = I.nx, ny = I.ny, nz = I.nz;
    const int x = (int)(s % nx);
    const long long t = s / nx;
    const int y = (int)(t % ny);
    const int z = (int)(t / ny);
    if (oG >= 0) {
      const Nbr nb = make_nbr(x, y, z, nx, ny, nz);
#pragma unroll
      for (int i = 0; i < 19; ++i) {
        const long long d = nb.off(-lat_c(i, 0), -lat_c(i, 1), -lat_c(i, 2));
        double fi = src[oG + i * N + s];
        if (SHIFT) fi -= lat_w(i) * (double)I.c.rho0;
        g_t[i * N + d] = (T)fi;
      }
    }
    if (oU >= 0)
      for (int a = 0; a < 3; ++a) u_t[a * N + s] = (T)src[oU + a * N + s];
    if (oQ >= 0)
      for (int k = 0; k < 5; ++k) q_t[k * N + s] = (T)src[oQ + k * N + s];
    if (oP >= 0) p_t[s] = (T)src[oP + s];
  }
}

// ---------------------------------------------------------------- FP64 reductions
// 12 sums per instance (see lbcad_obs).  Fixed-order block reduction with warp shuffles
// into partial[block][12]; k_obs_final sums the partials in block order.
template <typename T, bool SHIFT>
__global__ void __launch_bounds__(kObsBlock) k_obs_partial(InstDesc<T> I, double* __restrict__ partial) {
  double acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = 0.0;
  const long long N = I.N;
  const double two_pi = 6.283185307179586476925286766559;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N; s += (long long)gridDim.x * blockDim.x) {
    const int nx = I.nx, ny = I.ny, nz = I.nz;
    const int x = (int)(s % nx);
    const long long t = s / nx;
    const int y = (int)(t % ny);
    const int z = (int)(t / ny);
    const Nbr nb = make_nbr(x, y, z, nx, ny, nz);
#pragma unroll
    for (int i = 0; i < 19; ++i) {
      const long long src = nb.off(-lat_c(i, 0), -lat_c(i, 1), -lat_c(i, 2));
      double fi = (double)I.g_in[i * N + src];
      if (SHIFT) fi += lat_w(i) * (double)I.c.rho0;
      acc[0] += fi;
      if (lat_c(i, 0)) acc[2] += lat_c(i, 0) * fi;
      if (lat_c(i, 1)) acc[3] += lat_c(i, 1) * fi;
      if (lat_c(i, 2)) acc[4] += lat_c(i, 2) * fi;
    }
    const double p = (double)I.psi_in[s];
    acc[1] += p;
    const double pc = 0.5 * (1.0 + p);
    const int r[3] = {x, y, z};
    const int L[3] = {nx, ny, nz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double sn, cs;
      sincos(two_pi * (double)r[a] / (double)L[a], &sn, &cs);
      acc[5 + a] += pc * cs;
      acc[8 + a] += pc * sn;
    }
    acc[11] += pc;
  }
  __shared__ double sh[kObsBlock / 32][12];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    double v = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[wid][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < 12) {
    double v = 0.0;
    for (int w = 0; w < kObsBlock / 32; ++w) v += sh[w][threadIdx.x];
    partial[blockIdx.x * 12 + threadIdx.x] = v;
  }
}

static __global__ void k_obs_final(const double* __restrict__ partial, int nblocks, double* __restrict__ out) {
  if (threadIdx.x < 12) {
    double v = 0.0;
    for (int b = 0; b < nblocks; ++b) v += partial[b * 12 + threadIdx.x];
    out[threadIdx.x] = v;
  }
}

// ---------------------------------------------------------------- launchers
template <typename T, bool SHIFT>
cudaError_t Launch<T, SHIFT>::step(const InstDesc<T>* d_desc, int ninst, long long total_blocks, int bs,
                                   cudaStream_t s) {
  k_fields<T><<<(unsigned)total_blocks, bs, 0, s>>>(d_desc, ninst);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_update<T, SHIFT><<<(unsigned)total_blocks, bs, 0, s>>>(d_desc, ninst);
  return cudaGetLastError();
}

inline unsigned grid_for(long long N, int bs) {
  long long g = (N + bs - 1) / bs;
  if (g > 152 * 16) g = 152 * 16;
  return (unsigned)(g < 1 ? 1 : g);
}

template <typename T, bool SHIFT>
cudaError_t Launch<T, SHIFT>::get_fields(const InstDesc<T>& I, uint32_t mask, double* dst, cudaStream_t s) {
  long long o = 0, oG = -1, oR = -1, oU = -1, oQ = -1, oP = -1;
  if (mask & 1u) { oG = o; o += 19 * I.N; }
  if (mask & 2u) { oR = o; o += I.N; }
  if (mask & 4u) { oU = o; o += 3 * I.N; }
  if (mask & 8u) { oQ = o; o += 5 * I.N; }
  if (mask & 16u) { oP = o; o += I.N; }
  k_get_fields<T, SHIFT><<<grid_for(I.N, 256), 256, 0, s>>>(I, oG, oR, oU, oQ, oP, dst);
  return cudaGetLastError();
}

template <typename T, bool SHIFT>
cudaError_t Launch<T, SHIFT>::set_fields(const InstDesc<T>& I, uint32_t mask, const double* src, T* g_t, T* q_t,
                                         T* p_t, T* u_t, cudaStream_t s) {
  long long o = 0, oG = -1, oU = -1, oQ = -1, oP = -1;
  if (mask & 1u) { oG = o; o += 19 * I.N; }
  if (mask & 4u) { oU = o; o += 3 * I.N; }
  if (mask & 8u) { oQ = o; o += 5 * I.N; }
  if (mask & 16u) { oP = o; o += I.N; }
  k_set_fields<T, SHIFT><<<grid_for(I.N, 256), 256, 0, s>>>(I, oG, oU, oQ, oP, src, g_t, q_t, p_t, u_t);
  return cudaGetLastError();
}

template <typename T, bool SHIFT>
cudaError_t Launch<T, SHIFT>::observables(const InstDesc<T>& I, double* partial, int nblocks, double* out,
                                          cudaStream_t s) {
  k_obs_partial<T, SHIFT><<<nblocks, kObsBlock, 0, s>>>(I, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_obs_final<<<1, 32, 0, s>>>(partial, nblocks, out);
  return cudaGetLastError();
}

}  // namespace lbcad
