// lbcad_kernels.cuh -- CUDA kernels of the hybrid LB step, templated on the compute
// type T (float or double) and on SHIFT (populations stored as f_i - w_i rho0).
//
// The per-site device functions every path shares (stencils, local fields, order-parameter
// update, collision), the a6 pass, and the per-site kernels of the two cross-check paths.
// On the two-kernel path one step (Sec. 3 of Carenza, Gonnella & Negro) runs as:
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

// Periodic offsets of the sites at distance up to 2 along each axis (radius-2 stencils;
// every edge is >= 4, so one wrap suffices).
struct NbrR2 {
  int xo[5];
  int yo[5];
  long long zo[5];
  __device__ __forceinline__ long long off(int dx, int dy, int dz) const {
    return (long long)xo[dx + 2] + yo[dy + 2] + zo[dz + 2];
  }
};

__device__ __forceinline__ int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

__device__ __forceinline__ NbrR2 make_nbr_r2(int x, int y, int z, int nx, int ny, int nz) {
  NbrR2 n;
  const long long pl = (long long)nx * ny;
#pragma unroll
  for (int d = -2; d <= 2; ++d) {
    n.xo[d + 2] = wrap1(x + d, nx);
    n.yo[d + 2] = wrap1(y + d, ny) * nx;
    n.zo[d + 2] = wrap1(z + d, nz) * pl;
  }
  return n;
}

// Neighbour map of stencil set ST: 0 = isotropic D3Q19 (radius 1), 1 = fourth order (radius 2).
template <int ST>
__device__ __forceinline__ auto make_nbr_st(int x, int y, int z, int nx, int ny, int nz) {
  if constexpr (ST == 1) return make_nbr_r2(x, y, z, nx, ny, nz);
  else return make_nbr(x, y, z, nx, ny, nz);
}

// Full symmetric traceless tensor from the five stored components xx, xy, xz, yy, yz.
template <typename T>
__device__ __forceinline__ void full3(const T q[5], T Q[3][3]) {
  Q[0][0] = q[0]; Q[0][1] = q[1]; Q[0][2] = q[2];
  Q[1][0] = q[1]; Q[1][1] = q[3]; Q[1][2] = q[4];
  Q[2][0] = q[2]; Q[2][1] = q[4]; Q[2][2] = -q[0] - q[3];
}

// Two-lane values for packed arithmetic: float2 uses the f32x2 instructions (one issue
// slot for two lanes); other types fall back to two scalar operations.
template <typename T>
struct Vec2 {
  T x, y;
};
template <typename T>
__device__ __forceinline__ Vec2<T> v2(T a, T b) { return Vec2<T>{a, b}; }
template <typename T>
__device__ __forceinline__ Vec2<T> add2(Vec2<T> a, Vec2<T> b) { return Vec2<T>{a.x + b.x, a.y + b.y}; }
template <typename T>
__device__ __forceinline__ Vec2<T> sub2(Vec2<T> a, Vec2<T> b) { return Vec2<T>{a.x - b.x, a.y - b.y}; }
template <typename T>
__device__ __forceinline__ Vec2<T> fma2(Vec2<T> a, Vec2<T> b, Vec2<T> c) {
  return Vec2<T>{a.x * b.x + c.x, a.y * b.y + c.y};
}
template <typename T>
__device__ __forceinline__ Vec2<T> mul2(Vec2<T> a, Vec2<T> b) { return Vec2<T>{a.x * b.x, a.y * b.y}; }
__device__ __forceinline__ float2 f2(Vec2<float> a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ Vec2<float> v2f(float2 a) { return Vec2<float>{a.x, a.y}; }
template <>
__device__ __forceinline__ Vec2<float> add2(Vec2<float> a, Vec2<float> b) { return v2f(__fadd2_rn(f2(a), f2(b))); }
template <>
__device__ __forceinline__ Vec2<float> sub2(Vec2<float> a, Vec2<float> b) {
  return v2f(__ffma2_rn(f2(b), make_float2(-1.f, -1.f), f2(a)));  // a - b, one rounding
}
template <>
__device__ __forceinline__ Vec2<float> fma2(Vec2<float> a, Vec2<float> b, Vec2<float> c) {
  return v2f(__ffma2_rn(f2(a), f2(b), f2(c)));
}
template <>
__device__ __forceinline__ Vec2<float> mul2(Vec2<float> a, Vec2<float> b) { return v2f(__fmul2_rn(f2(a), f2(b))); }

// Gradient (1/12)[2 D_face + signed edge pairs] from opposite-pair differences D[i] =
// f(c_i) - f(c_{i+1}), two fields at once.
template <typename T>
__device__ __forceinline__ void grad2_from_pairs(const Vec2<T> D[19], Vec2<T> g[3]) {
  const Vec2<T> k2 = v2(T(2), T(2)), k12 = v2(T(1.0 / 12.0), T(1.0 / 12.0));
  g[0] = mul2(fma2(D[1], k2, add2(add2(D[7], D[9]), add2(D[11], D[13]))), k12);
  g[1] = mul2(fma2(D[3], k2, add2(sub2(D[7], D[9]), add2(D[15], D[17]))), k12);
  g[2] = mul2(fma2(D[5], k2, add2(sub2(D[11], D[13]), sub2(D[15], D[17]))), k12);
}

// Stress and chemical potential as five pairs, the unit of the tiles in shared memory:
// pair j of a site holds (sigma_xb, sigma_yb) for j = b = 0, 1, 2, (sigma_zx, sigma_zy) for
// j = 3 and (sigma_zz, mu) for j = 4.  sig_pair(c) = j and sig_lane(c) = lane of sigma_c
// (c = 3a + b); mu sits in pair 4, lane 1.
__host__ __device__ constexpr int sig_pair(int c) { return c < 6 ? c % 3 : (c < 8 ? 3 : 4); }
__host__ __device__ constexpr int sig_lane(int c) { return c < 6 ? c / 3 : (c < 8 ? c - 6 : 0); }
// the two stress components of pair j (the second is -1 for mu)
__host__ __device__ constexpr int pair_c0(int j) { return j < 3 ? j : (j == 3 ? 6 : 8); }
__host__ __device__ constexpr int pair_c1(int j) { return j < 3 ? j + 3 : (j == 3 ? 7 : -1); }

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
  // Q.Q is symmetric: six products
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
  // curl: C_ab = eps_amn d_m Q_nb, and its symmetric part CC = C + C^T
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
    for (int j = i; j < 3; ++j) {
      CC[i][j] = C[i][j] + C[j][i];
      CC[j][i] = CC[i][j];
    }
  const T g2 = dp[0] * dp[0] + dp[1] * dp[1] + dp[2] * dp[2];
  const T Ac = c.A0 * chi;
  const T Kq = T(2) * c.K * c.q0;
  const T lin = -c.A0 * (T(1) - chi / T(3)) - Ac * trQ2 - Kq * T(2) * c.q0;
  const T iso = (Ac * trQ2 - c.W * g2) / T(3);
  // H = -dF/dQ (traceless symmetric by construction: tr CC = 0 for symmetric Q)
  const int I5[5] = {0, 0, 0, 1, 1};
  const int J5[5] = {0, 1, 2, 1, 2};
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int i = I5[k], j = J5[k];
    T h = lin * Q[i][j] + Ac * QQ[i][j] + c.K * lapq[k] - Kq * CC[i][j] - c.W * dp[i] * dp[j];
    if (i == j) h -= iso;
    H[k] = h;
  }
  T Hf[3][3];
  full3(H, Hf);

  // mu = dF/dpsi
  const T Qh = Q[0][0] * hp[0] + Q[1][1] * hp[1] + Q[2][2] * hp[2] +
               T(2) * (Q[0][1] * hp[3] + Q[0][2] * hp[4] + Q[1][2] * hp[5]);
  T divQdp = T(0);
#pragma unroll
  for (int b = 0; b < 3; ++b) divQdp += (dQ[0][0][b] + dQ[1][1][b] + dQ[2][2][b]) * dp[b];
  const T psi2 = psi * psi;
  mu = psi * (c.b * psi2 - c.a) - c.kphi * lapp + c.A0 * c.chis * (trQ2 * (T(0.25) * trQ2 - T(1) / T(6)) - trQ3 / T(3)) -
       T(2) * c.W * (divQdp + Qh);

  // Gram matrix of the Q derivatives (symmetric), Q:curl Q, Q.grad psi
  T G[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = a; b < 3; ++b) {
      const T s = dQ[a][0][0] * dQ[b][0][0] + dQ[a][1][1] * dQ[b][1][1] + dQ[a][2][2] * dQ[b][2][2] +
                  T(2) * (dQ[a][0][1] * dQ[b][0][1] + dQ[a][0][2] * dQ[b][0][2] + dQ[a][1][2] * dQ[b][1][2]);
      G[a][b] = s;
      G[b][a] = s;
    }
  const T QC = Q[0][0] * C[0][0] + Q[1][1] * C[1][1] + Q[2][2] * C[2][2] + Q[0][1] * CC[0][1] +
               Q[0][2] * CC[0][2] + Q[1][2] * CC[1][2];
  T Qdp[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) Qdp[i] = Q[i][0] * dp[0] + Q[i][1] * dp[1] + Q[i][2] * dp[2];
  const T anch = dp[0] * Qdp[0] + dp[1] * Qdp[1] + dp[2] * Qdp[2];
  const T fden = psi2 * (T(0.25) * c.b * psi2 - T(0.5) * c.a) + T(0.5) * c.kphi * g2 +
                 c.A0 * (T(0.5) * (T(1) - chi / T(3)) * trQ2 - chi / T(3) * trQ3 + chi / T(4) * trQ2 * trQ2) +
                 T(0.5) * c.K * (G[0][0] + G[1][1] + G[2][2]) + Kq * QC + Kq * c.q0 * trQ2 + c.W * anch;
  const T P0 = psi * mu - fden;

  // reactive and active parts: with (HQ)_ab = (QH)_ba,
  //   -xi (HQ~ + Q~H) + 2 xi Q~ tr(QH) + QH - HQ - zeta phi_c Q
  //   = (1 - xi) QH - (1 + xi) HQ - (2 xi/3) H + (2 xi tr(QH) - zeta phi_c) Q + (2 xi/3) tr(QH) I
  T QH[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) QH[i][j] = Q[i][0] * Hf[0][j] + Q[i][1] * Hf[1][j] + Q[i][2] * Hf[2][j];
  const T trQH = QH[0][0] + QH[1][1] + QH[2][2];
  const T phic = T(0.5) * (T(1) + psi);
  const T cQ = T(2) * c.xi * trQH - c.zeta * phic;
  const T cI = T(2) * c.xi / T(3) * trQH - P0;
  const T cH = -T(2) * c.xi / T(3);
  const T cP = T(1) - c.xi, cM = -(T(1) + c.xi);
  T wv[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) wv[b] = c.kphi * dp[b] + T(2) * c.W * Qdp[b];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    // v_b = eps_bgm (dQ_a Q)_gm: the axial vector of the antisymmetric part of dQ_a Q
    T v[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int g = (b + 1) % 3, m = (b + 2) % 3;
      v[b] = dQ[a][g][0] * Q[0][m] + dQ[a][g][1] * Q[1][m] + dQ[a][g][2] * Q[2][m] -
             (dQ[a][m][0] * Q[0][g] + dQ[a][m][1] * Q[1][g] + dQ[a][m][2] * Q[2][g]);
    }
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      T s = cQ * Q[a][b] + cP * QH[a][b] + cM * QH[b][a] + cH * Hf[a][b] - c.K * G[a][b] - Kq * v[b] - dp[a] * wv[b];
      if (a == b) s += cI;
      sig[3 * a + b] = s;
    }
  }
}

// ---------------------------------------------------------------- shared per-site pieces
// Both step paths (two kernels through global memory, one fused kernel through shared
// memory tiles) evaluate their stencils with the functions below, in the same order and
// with the same arithmetic, through an accessor A that returns neighbour values:
//   A::q(k, cx, cy, cz), A::psi(cx, cy, cz)            (gather_fields)
//   A::sig(k, ...), A::mu(...), A::u(a, ...), q, psi   (gather_update)
// With cx, cy, cz compile-time constants after unrolling, a shared-memory accessor
// turns every neighbour read into one load at an immediate offset.
//
// D3Q19 velocities come in opposite pairs (i, i+1) for odd i, so the isotropic gradient
// 3 Sum_i w_i c_i f(x + c_i) is (1/12) Sum_pairs c_i (f_i - f_{i+1}) (x2 for faces):
//   d_x = [2 D1 + D7 + D9 + D11 + D13]/12,  d_y = [2 D3 + D7 - D9 + D15 + D17]/12,
//   d_z = [2 D5 + D11 - D13 + D15 - D17]/12,  D_i = f(x + c_i) - f(x + c_{i+1}).
// Laplacians are sums of differences to the centre value (Sum_i w_i c_i = 0), which
// keeps them free of cancellation in FP32.

template <typename T>
__device__ __forceinline__ void grad_from_pairs(const T D[19], T g[3]) {
  g[0] = (T(2) * D[1] + D[7] + D[9] + D[11] + D[13]) * T(1.0 / 12.0);
  g[1] = (T(2) * D[3] + D[7] - D[9] + D[15] + D[17]) * T(1.0 / 12.0);
  g[2] = (T(2) * D[5] + D[11] - D[13] + D[15] - D[17]) * T(1.0 / 12.0);
}

// Laplacian from differences to the centre: (1/3) Sum_faces d + (1/6) Sum_edges d.
template <typename T>
__device__ __forceinline__ T lap_from_diffs(const T d[19]) {
  const T sf = (d[1] + d[2]) + (d[3] + d[4]) + (d[5] + d[6]);
  const T se = ((d[7] + d[8]) + (d[9] + d[10])) + ((d[11] + d[12]) + (d[13] + d[14])) +
               ((d[15] + d[16]) + (d[17] + d[18]));
  return (T(2) * sf + se) * T(1.0 / 6.0);
}

// a1: gradient and Laplacian of the five Q components and psi, and the Hessian of psi
// (three-point differences on the diagonal, four corners off it).  The six fields are
// taken in pairs (Q_xx, Q_xy), (Q_xz, Q_yy), (Q_yz, psi) through A::pair(j, ...), so one
// two-lane operation advances two fields.
template <typename T, class A>
__device__ __forceinline__ void gather_fields(const A& acc, T q0[5], T& p0, T dq[3][5], T lapq[5], T dp[3],
                                              T& lapp, T hp[6]) {
  using V = Vec2<T>;
  const V k2 = v2(T(2), T(2)), k6 = v2(T(1.0 / 6.0), T(1.0 / 6.0));
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    V f[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) f[i] = acc.pair(j, lat_c(i, 0), lat_c(i, 1), lat_c(i, 2));
    V d[19], D[19];
#pragma unroll
    for (int i = 1; i < 19; ++i) d[i] = sub2(f[i], f[0]);
#pragma unroll
    for (int i = 1; i < 19; i += 2) D[i] = sub2(d[i], d[i + 1]);
    V g[3];
    grad2_from_pairs<T>(D, g);
    // Laplacian from differences to the centre: (1/3) faces + (1/6) edges
    const V sf = add2(add2(add2(d[1], d[2]), add2(d[3], d[4])), add2(d[5], d[6]));
    const V se = add2(add2(add2(add2(d[7], d[8]), add2(d[9], d[10])), add2(add2(d[11], d[12]), add2(d[13], d[14]))),
                      add2(add2(d[15], d[16]), add2(d[17], d[18])));
    const V lp = mul2(fma2(sf, k2, se), k6);
    const int k0 = 2 * j;
    q0[k0] = f[0].x;
    lapq[k0] = lp.x;
#pragma unroll
    for (int a = 0; a < 3; ++a) dq[a][k0] = g[a].x;
    if (j < 2) {
      q0[k0 + 1] = f[0].y;
      lapq[k0 + 1] = lp.y;
#pragma unroll
      for (int a = 0; a < 3; ++a) dq[a][k0 + 1] = g[a].y;
    } else {
      p0 = f[0].y;
      lapp = lp.y;
#pragma unroll
      for (int a = 0; a < 3; ++a) dp[a] = g[a].y;
      hp[0] = d[1].y + d[2].y;
      hp[1] = d[3].y + d[4].y;
      hp[2] = d[5].y + d[6].y;
      hp[3] = T(0.25) * ((d[7].y + d[8].y) - (d[9].y + d[10].y));
      hp[4] = T(0.25) * ((d[11].y + d[12].y) - (d[13].y + d[14].y));
      hp[5] = T(0.25) * ((d[15].y + d[16].y) - (d[17].y + d[18].y));
    }
  }
}

// a3 (divergence): F_a = d_b sigma_ab from opposite-pair differences of sigma, through the
// stress pairs A::spair(j, ...): (F_x, F_y) from pairs 0-2 two lanes at a time, F_z from
// pair 3 (sigma_zx, sigma_zy) and lane 0 of pair 4 (sigma_zz).
template <typename T, class A>
__device__ __forceinline__ void gather_force(const A& acc, T F[3]) {
  using V = Vec2<T>;
  V a2 = v2(T(0), T(0)), a1 = v2(T(0), T(0));
#pragma unroll
  for (int b = 0; b < 3; ++b) {
#pragma unroll
    for (int i = 1; i < 19; i += 2) {
      const int cb = lat_c(i, b);
      if (cb == 0) continue;
      const V D = sub2(acc.spair(b, lat_c(i, 0), lat_c(i, 1), lat_c(i, 2)),
                       acc.spair(b, lat_c(i + 1, 0), lat_c(i + 1, 1), lat_c(i + 1, 2)));
      if (lat_c2(i) == 1) a2 = cb > 0 ? add2(a2, D) : sub2(a2, D);
      else a1 = cb > 0 ? add2(a1, D) : sub2(a1, D);
    }
  }
  const V fxy = mul2(fma2(a2, v2(T(2), T(2)), a1), v2(T(1.0 / 12.0), T(1.0 / 12.0)));
  F[0] = fxy.x;
  F[1] = fxy.y;
  T z2 = T(0), z1 = T(0);
#pragma unroll
  for (int i = 1; i < 19; i += 2) {
    const int cx = lat_c(i, 0), cy = lat_c(i, 1), cz = lat_c(i, 2);
    const bool face = lat_c2(i) == 1;
    if (cx || cy) {
      const V D = sub2(acc.spair(3, cx, cy, cz), acc.spair(3, -cx, -cy, -cz));
      if (cx) {
        const T d = cx > 0 ? D.x : -D.x;
        if (face) z2 += d; else z1 += d;
      }
      if (cy) {
        const T d = cy > 0 ? D.y : -D.y;
        if (face) z2 += d; else z1 += d;
      }
    }
    if (cz) {
      const T Dz = acc.spair(4, cx, cy, cz).x - acc.spair(4, -cx, -cy, -cz).x;
      const T d = cz > 0 ? Dz : -Dz;
      if (face) z2 += d; else z1 += d;
    }
  }
  F[2] = (T(2) * z2 + z1) * T(1.0 / 12.0);
}

// The stencils of a4: lap mu, W_ab = d_b u_a, and the face values of Q, psi and u for the
// upwind terms (face slot 2a: +e_a, 2a+1: -e_a).
template <typename T, class A>
__device__ __forceinline__ void gather_op(const A& acc, T& lapmu, T Wg[3][3], T q0[5], T qf[6][5], T& p0, T pf[6],
                                          T u0[3], T uf[6]) {
  // lap mu (lane 1 of stress pair 4, so that the loads are shared with the force)
  {
    T d[19];
    const T m0 = acc.spair(4, 0, 0, 0).y;
#pragma unroll
    for (int i = 1; i < 19; ++i) d[i] = acc.spair(4, lat_c(i, 0), lat_c(i, 1), lat_c(i, 2)).y - m0;
    lapmu = lap_from_diffs(d);
  }
  // grad u and the axial face velocities: (u_x, u_y) as pairs, u_z alone
  {
    using V = Vec2<T>;
    V f[19], D[19], g[3];
#pragma unroll
    for (int i = 0; i < 19; ++i) f[i] = acc.upair(lat_c(i, 0), lat_c(i, 1), lat_c(i, 2));
#pragma unroll
    for (int i = 1; i < 19; i += 2) D[i] = sub2(f[i], f[i + 1]);
    grad2_from_pairs<T>(D, g);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      Wg[0][b] = g[b].x;
      Wg[1][b] = g[b].y;
    }
    u0[0] = f[0].x;
    u0[1] = f[0].y;
    uf[0] = f[1].x;
    uf[1] = f[2].x;
    uf[2] = f[3].y;
    uf[3] = f[4].y;
  }
  {
    T f[19], D[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) f[i] = acc.u(2, lat_c(i, 0), lat_c(i, 1), lat_c(i, 2));
#pragma unroll
    for (int i = 1; i < 19; i += 2) D[i] = f[i] - f[i + 1];
    grad_from_pairs(D, Wg[2]);
    u0[2] = f[0];
    uf[4] = f[5];
    uf[5] = f[6];
  }
  // Q and psi at the centre and the six faces, as the field pairs (Q_xx, Q_xy), (Q_xz, Q_yy),
  // (Q_yz, psi) of A::pair
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    const int cx = lat_c(i, 0), cy = lat_c(i, 1), cz = lat_c(i, 2);
    T* qd = i ? qf[i - 1] : q0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const Vec2<T> v = acc.pair(j, cx, cy, cz);
      qd[2 * j] = v.x;
      if (j < 2) qd[2 * j + 1] = v.y;
      else if (i) pf[i - 1] = v.y;
      else p0 = v.y;
    }
  }
}

// a3 + the stencils of a4, for the one-pass step.
template <typename T, class A>
__device__ __forceinline__ void gather_update(const A& acc, T F[3], T& lapmu, T Wg[3][3], T q0[5], T qf[6][5],
                                              T& p0, T pf[6], T u0[3], T uf[6]) {
  gather_force<T>(acc, F);
  gather_op<T>(acc, lapmu, Wg, q0, qf, p0, pf, u0, uf);
}

// a4 at one site: Beris-Edwards update of Q (Eq. 2) and Cahn-Hilliard update of psi
// (Eq. 1) with the advecting velocity u0/uf (and its gradient Wg).  RHS = false gives the
// Euler step Q + R(Q), RHS = true the right-hand side R(Q) alone (for the Heun stages).
template <typename T, bool RHS>
__device__ __forceinline__ void op_update(const Coef<T>& c, T lapmu, const T Wg[3][3], const T q0[5],
                                          const T qf[6][5], T p0, const T pf[6], const T u0[3], const T uf[6],
                                          const T Hs[5], T qn[5], T& pn) {
  T adv[5] = {T(0), T(0), T(0), T(0), T(0)};
  T divJ = T(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int ip = 2 * a, im = 2 * a + 1;
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
  // co-rotation S = (xi D + Om)(Q + I/3) + (Q + I/3)(xi D - Om) - 2 xi tr(QW)(Q + I/3), with
  // D, Om the symmetric and antisymmetric parts of W.  With M = xi D + Om, (xi D - Om) = M^T, so
  // S = P + P^T - 2 xi tr(QW)(Q + I/3) for P = M (Q + I/3); it is projected to its traceless part
  // (its trace is 2 xi tr(D)/3).  M_ij = (xi + 1)/2 W_ij + (xi - 1)/2 W_ji.
  const T mp = T(0.5) * (c.xi + T(1)), mm = T(0.5) * (c.xi - T(1));
  T M[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) M[i][j] = mp * Wg[i][j] + mm * Wg[j][i];
  T Qt[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Qt[i][j] = i == j ? Q[i][j] + T(1.0 / 3.0) : Q[i][j];
  T trQW = T(0);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) trQW += Q[i][j] * Wg[j][i];
  const T trD = Wg[0][0] + Wg[1][1] + Wg[2][2];
  const T cq = -T(2) * c.xi * trQW;
  const T cdiag = -(T(2) * c.xi / T(9)) * trD;
  auto P = [&](int i, int j) { return M[i][0] * Qt[0][j] + M[i][1] * Qt[1][j] + M[i][2] * Qt[2][j]; };
  // The increments are summed first and added to Q and psi once: every addition at the
  // magnitude of the field rounds to its storage resolution, and three of them per step
  // (Q - adv, + S, + Gamma H) added half again to the error that FP32 storage alone causes.
  const int I5[5] = {0, 0, 0, 1, 1};
  const int J5[5] = {0, 1, 2, 1, 2};
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int i = I5[k], j = J5[k];
    T S = (i == j ? T(2) * P(i, i) : P(i, j) + P(j, i)) + cq * Qt[i][j];
    if (i == j) S += cdiag;
    const T inc = fma(c.gammaQ, Hs[k], S - adv[k]);
    qn[k] = RHS ? inc : q0[k] + inc;
  }
  const T pinc = fma(c.M, lapmu, -divJ);
  pn = RHS ? pinc : p0 + pinc;
}

// a5 at one site: moments of the pulled populations g and the force F, then BGK + Guo
// collision (Eqs. 6-8); g is overwritten with the post-collision values, u = velocity.
// The equilibrium and forcing terms of opposite velocities c and -c share their even part.
// mom (optional): the site's share of the conserved sums of the new state, mom[0] = mass
// (minus rho0 when SHIFT) and mom[1..3] = post-collision momentum j + F.
template <typename T, bool SHIFT, class V = VelD3Q19>
__device__ __forceinline__ void lb_collide(const Coef<T>& c, const T F[3], T g[V::Q], T u[3], T* mom = nullptr) {
  // moments from opposite pairs
  T m0 = g[0];
  T j[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int i = 1; i < V::Q; i += 2) {
    m0 += g[i] + g[i + 1];
    const T dg = g[i] - g[i + 1];
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (V::c(i, a)) j[a] += V::c(i, a) > 0 ? dg : -dg;
  }
  const T rho = SHIFT ? (c.rho0 + m0) : m0;
  const T rinv = T(1) / rho;
  // every product-sum below is an explicit fma: the collision then rounds identically in every
  // kernel that inlines it, whatever the compiler would contract
#pragma unroll
  for (int a = 0; a < 3; ++a) u[a] = fma(T(0.5), F[a], j[a]) * rinv;
  if (mom) {
    mom[0] = m0;
#pragma unroll
    for (int a = 0; a < 3; ++a) mom[1 + a] = j[a] + F[a];
  }
  const T u2 = fma(u[2], u[2], fma(u[1], u[1], u[0] * u[0]));
  const T uF = fma(u[2], F[2], fma(u[1], F[1], u[0] * F[0]));
  // BGK + Guo as g' = (1 - om) g + om f_eq + F_i, with the equilibrium
  // w rho (1 + 3 cu + 4.5 cu^2 - 1.5 u^2) (shifted: minus w rho0) and the Guo term
  // guo w (3 (c - u).F + 9 (c.u)(c.F)).  For the pair (c, -c) the new values are
  // (1 - om) g_(+-) + (X +- Y), with the even part X = om w (base + 4.5 rho cu^2) + guo w
  // (9 cu cF - 3 uF) and the odd part Y = 3 om w rho cu + 3 guo w cF; their coefficients depend
  // on the weight class only, so each class forms them once.
  const T base = fma(T(-1.5) * rho, u2, SHIFT ? m0 : rho);
  const T om = c.tau_inv;
  const T omc = T(1) - om;
  const T r45 = T(4.5) * rho;
  const T r3 = T(3) * rho;
  {
    const T w = T(V::w(0));
    g[0] = fma(omc, g[0], fma(om * w, base, (T(-3) * c.guo * w) * uF));
  }
#pragma unroll
  for (int i = 1; i < V::Q; i += 2) {
    const T w = T(V::w(i));
    const T omw = om * w, gw = c.guo * w;
    const T cu = T(V::c(i, 0)) * u[0] + T(V::c(i, 1)) * u[1] + T(V::c(i, 2)) * u[2];
    const T cF = T(V::c(i, 0)) * F[0] + T(V::c(i, 1)) * F[1] + T(V::c(i, 2)) * F[2];
    const T X = fma(omw * r45, cu * cu, fma(omw, base, fma((T(9) * gw) * cu, cF, (T(-3) * gw) * uF)));
    const T Y = fma(omw * r3, cu, (T(3) * gw) * cF);
    const T gp = g[i], gm = g[i + 1];
    g[i] = fma(omc, gp, X + Y);
    g[i + 1] = fma(omc, gm, X - Y);
  }
}

// a5 in the form of Eqs. 9-11 at one site: the equilibrium carries the symmetric stress,
//   f_eq_i = w_i [rho + 3 rho c.u + (9/2)(c c - I/3) : (rho u u - sigma^S)],
// the antisymmetric stress enters as F_i = 3 w_i c . FA with FA = div sigma^A (moments 0, FA,
// 0: Eq. 10), rho u = sum f c (Eq. 8), f* = f - (f - f_eq)/tau + F_i (Eq. 7).  sig is the full
// stress at the site (9, row-major).  Opposite velocities share the even part of f_eq.
template <typename T, bool SHIFT, class V>
__device__ __forceinline__ void lb_collide_stress(const Coef<T>& c, const T FA[3], const T sig[9], T g[V::Q],
                                                  T u[3], T* mom = nullptr) {
  T m0 = g[0];
  T j[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int i = 1; i < V::Q; i += 2) {
    m0 += g[i] + g[i + 1];
    const T dg = g[i] - g[i + 1];
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (V::c(i, a)) j[a] += V::c(i, a) > 0 ? dg : -dg;
  }
  const T rho = SHIFT ? (c.rho0 + m0) : m0;
  const T rinv = T(1) / rho;
#pragma unroll
  for (int a = 0; a < 3; ++a) u[a] = j[a] * rinv;
  if (mom) {  // as in lb_collide: the forcing adds FA to the momentum (Eq. 10)
    mom[0] = m0;
#pragma unroll
    for (int a = 0; a < 3; ++a) mom[1 + a] = j[a] + FA[a];
  }
  // Pi = rho u u - sigma^S (symmetric: xx, yy, zz, xy, xz, yz)
  const T Pxx = rho * u[0] * u[0] - sig[0], Pyy = rho * u[1] * u[1] - sig[4], Pzz = rho * u[2] * u[2] - sig[8];
  const T Pxy = rho * u[0] * u[1] - T(0.5) * (sig[1] + sig[3]);
  const T Pxz = rho * u[0] * u[2] - T(0.5) * (sig[2] + sig[6]);
  const T Pyz = rho * u[1] * u[2] - T(0.5) * (sig[5] + sig[7]);
  const T tr3 = (Pxx + Pyy + Pzz) * T(1.0 / 3.0);
  // even part: w (rho + 4.5 (c.Pi.c - tr Pi/3)), minus w rho0 when shifted
  const T base = SHIFT ? m0 : rho;
  const T om = c.tau_inv;
  {
    const T w = T(V::w(0));
    const T geq = w * (base - T(4.5) * tr3);
    g[0] = g[0] - (g[0] - geq) * om;
  }
#pragma unroll
  for (int i = 1; i < V::Q; i += 2) {
    const T w = T(V::w(i));
    const int cx = V::c(i, 0), cy = V::c(i, 1), cz = V::c(i, 2);
    const T cPc = T(cx * cx) * Pxx + T(cy * cy) * Pyy + T(cz * cz) * Pzz +
                  T(2 * cx * cy) * Pxy + T(2 * cx * cz) * Pxz + T(2 * cy * cz) * Pyz;
    const T cu = T(cx) * u[0] + T(cy) * u[1] + T(cz) * u[2];
    const T cF = T(cx) * FA[0] + T(cy) * FA[1] + T(cz) * FA[2];
    const T Aeq = w * (base + T(4.5) * (cPc - tr3));
    const T Beq = w * T(3) * rho * cu;
    const T Ef = T(3) * w * cF;
    const T gp = g[i], gm = g[i + 1];
    g[i] = gp - (gp - (Aeq + Beq)) * om + Ef;
    g[i + 1] = gm - (gm - (Aeq - Beq)) * om - Ef;
  }
}

// a4 + a5 of the one-pass step: Euler update of Q and psi with the velocity of the
// previous step, and the collision of the pulled populations.
template <typename T, bool SHIFT>
__device__ __forceinline__ void update_math(const Coef<T>& c, const T F[3], T lapmu, const T Wg[3][3],
                                            const T q0[5], const T qf[6][5], T p0, const T pf[6], const T u0[3],
                                            const T uf[6], const T Hs[5], T g[19], T qn[5], T& pn, T u[3]) {
  op_update<T, false>(c, lapmu, Wg, q0, qf, p0, pf, u0, uf, Hs, qn, pn);
  lb_collide<T, SHIFT>(c, F, g, u);
}

// Neighbour reads straight from global memory with periodic wrap (two-kernel path).
template <typename T, class NB = Nbr>
struct GlobalAcc {
  const T* q_;
  const T* ps;
  const T* sg;
  const T* mu_;
  const T* u_;
  long long N;
  NB nb;
  __device__ __forceinline__ T q(int k, int cx, int cy, int cz) const { return ld(q_ + k * N + nb.off(cx, cy, cz)); }
  __device__ __forceinline__ T psi(int cx, int cy, int cz) const { return ld(ps + nb.off(cx, cy, cz)); }
  __device__ __forceinline__ T sig(int k, int cx, int cy, int cz) const { return ld(sg + k * N + nb.off(cx, cy, cz)); }
  __device__ __forceinline__ T mu(int cx, int cy, int cz) const { return ld(mu_ + nb.off(cx, cy, cz)); }
  __device__ __forceinline__ T u(int a, int cx, int cy, int cz) const { return ld(u_ + a * N + nb.off(cx, cy, cz)); }
  // fields (2j, 2j+1) of the order (Q_xx, Q_xy, Q_xz, Q_yy, Q_yz, psi)
  __device__ __forceinline__ Vec2<T> pair(int j, int cx, int cy, int cz) const {
    const long long o = nb.off(cx, cy, cz);
    return Vec2<T>{ld(q_ + (2 * j) * N + o), j < 2 ? ld(q_ + (2 * j + 1) * N + o) : ld(ps + o)};
  }
  // stress pair j (see sig_pair) and the velocity pair (u_x, u_y)
  __device__ __forceinline__ Vec2<T> spair(int j, int cx, int cy, int cz) const {
    const long long o = nb.off(cx, cy, cz);
    return Vec2<T>{ld(sg + pair_c0(j) * N + o), j == 4 ? ld(mu_ + o) : ld(sg + pair_c1(j) * N + o)};
  }
  __device__ __forceinline__ Vec2<T> upair(int cx, int cy, int cz) const {
    const long long o = nb.off(cx, cy, cz);
    return Vec2<T>{ld(u_ + o), ld(u_ + N + o)};
  }
};

// ---------------------------------------------------------------- radius-2 stencils
// Fourth-order central differences along the axes (the other reading of "fourth-order
// accurate stencils", Sec. 3):
//   d_a f = [8 (f(+1) - f(-1)) - (f(+2) - f(-2))] / 12,
//   d_aa f = [16 (f(+1) + f(-1)) - (f(+2) + f(-2)) - 30 f(0)] / 12 (summed as differences to
//   f(0)), d_a d_b f = d_a of d_b f (16 points), the Laplacian = sum of the d_aa.
// F(dx, dy, dz) returns the field at the offset.
template <typename T, class F>
__device__ __forceinline__ void r2_axis(const F& f, T c, int a, T& d1, T& d2) {
  const int ex = a == 0, ey = a == 1, ez = a == 2;
  const T m2 = f(-2 * ex, -2 * ey, -2 * ez), m1 = f(-ex, -ey, -ez), p1 = f(ex, ey, ez), p2 = f(2 * ex, 2 * ey, 2 * ez);
  d1 = (T(8) * (p1 - m1) - (p2 - m2)) * T(1.0 / 12.0);
  // as differences to the centre, so that FP32 does not cancel terms of size 30 f
  d2 = (T(16) * ((p1 - c) + (m1 - c)) - ((p2 - c) + (m2 - c))) * T(1.0 / 12.0);
}

template <typename T, class F>
__device__ __forceinline__ T r2_mixed(const F& f, int a, int b) {
  const T w[5] = {T(1.0 / 12.0), T(-8.0 / 12.0), T(0), T(8.0 / 12.0), T(-1.0 / 12.0)};
  T s = T(0);
#pragma unroll
  for (int i = -2; i <= 2; ++i) {
    if (i == 0) continue;
    T r = T(0);
#pragma unroll
    for (int j = -2; j <= 2; ++j) {
      if (j == 0) continue;
      const int dx = (a == 0 ? i : 0) + (b == 0 ? j : 0);
      const int dy = (a == 1 ? i : 0) + (b == 1 ? j : 0);
      const int dz = (a == 2 ? i : 0) + (b == 2 ? j : 0);
      r += w[j + 2] * f(dx, dy, dz);
    }
    s += w[i + 2] * r;
  }
  return s;
}

// a1 with the radius-2 set: the same outputs as gather_fields.
template <typename T, class A>
__device__ __forceinline__ void gather_fields_r2(const A& acc, T q0[5], T& p0, T dq[3][5], T lapq[5], T dp[3],
                                                 T& lapp, T hp[6]) {
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    auto f = [&](int dx, int dy, int dz) { return acc.q(k, dx, dy, dz); };
    const T c = f(0, 0, 0);
    q0[k] = c;
    T l = T(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      T d1, d2;
      r2_axis<T>(f, c, a, d1, d2);
      dq[a][k] = d1;
      l += d2;
    }
    lapq[k] = l;
  }
  auto fp = [&](int dx, int dy, int dz) { return acc.psi(dx, dy, dz); };
  p0 = fp(0, 0, 0);
  T l = T(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    T d1, d2;
    r2_axis<T>(fp, p0, a, d1, d2);
    dp[a] = d1;
    hp[a] = d2;
    l += d2;
  }
  lapp = l;
  hp[3] = r2_mixed<T>(fp, 0, 1);
  hp[4] = r2_mixed<T>(fp, 0, 2);
  hp[5] = r2_mixed<T>(fp, 1, 2);
}

// a3 with the radius-2 set: F_a = sum_b d_b sigma_ab.
template <typename T, class A>
__device__ __forceinline__ void gather_force_r2(const A& acc, T F[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    T s = T(0);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int k = 3 * a + b;
      auto f = [&](int dx, int dy, int dz) { return acc.sig(k, dx, dy, dz); };
      T d1, d2;
      r2_axis<T>(f, T(0), b, d1, d2);
      s += d1;
    }
    F[a] = s;
  }
}

// The stencils of a4 with the radius-2 set; the upwind faces stay at distance 1.
template <typename T, class A>
__device__ __forceinline__ void gather_op_r2(const A& acc, T& lapmu, T Wg[3][3], T q0[5], T qf[6][5], T& p0,
                                             T pf[6], T u0[3], T uf[6]) {
  {
    auto f = [&](int dx, int dy, int dz) { return acc.mu(dx, dy, dz); };
    const T c = f(0, 0, 0);
    T l = T(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      T d1, d2;
      r2_axis<T>(f, c, a, d1, d2);
      l += d2;
    }
    lapmu = l;
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    auto f = [&](int dx, int dy, int dz) { return acc.u(a, dx, dy, dz); };
    u0[a] = f(0, 0, 0);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      T d1, d2;
      r2_axis<T>(f, u0[a], b, d1, d2);
      Wg[a][b] = d1;
    }
    uf[2 * a] = f(a == 0, a == 1, a == 2);
    uf[2 * a + 1] = f(-(a == 0), -(a == 1), -(a == 2));
  }
#pragma unroll
  for (int i = 1; i < 7; ++i) {
    const int cx = lat_c(i, 0), cy = lat_c(i, 1), cz = lat_c(i, 2);
#pragma unroll
    for (int k = 0; k < 5; ++k) qf[i - 1][k] = acc.q(k, cx, cy, cz);
    pf[i - 1] = acc.psi(cx, cy, cz);
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) q0[k] = acc.q(k, 0, 0, 0);
  p0 = acc.psi(0, 0, 0);
}

// ---------------------------------------------------------------- k_fields
// H, mu and sigma of (q_in, psi_in) into the scratch; with PRED, H and mu of the Heun
// predicted state qp into the (then free) sigma scratch: H at sig[0..5N), mu at sig[5N..6N).
template <typename T, bool PRED = false, int ST = 0>
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
  GlobalAcc<T, decltype(make_nbr_st<ST>(0, 0, 0, 4, 4, 4))> acc;
  acc.q_ = PRED ? I.qp : I.q_in;
  acc.ps = PRED ? I.qp + 5 * N : I.psi_in;
  acc.N = N;
  acc.nb = make_nbr_st<ST>(x, y, z, nx, ny, nz);
  T q0[5], p0, dq[3][5], lapq[5], dp[3], lapp, hp[6];
  if constexpr (ST == 1) gather_fields_r2<T>(acc, q0, p0, dq, lapq, dp, lapp, hp);
  else gather_fields<T>(acc, q0, p0, dq, lapq, dp, lapp, hp);
  T H[5], sig[9], mu;
  local_fields<T>(I.c, q0, p0, dq, lapq, dp, lapp, hp, H, mu, sig);
  if constexpr (PRED) {
#pragma unroll
    for (int k = 0; k < 5; ++k) I.sig[k * N + s] = H[k];
    I.sig[5 * N + s] = mu;
  } else {
#pragma unroll
    for (int k = 0; k < 5; ++k) I.H[k * N + s] = H[k];
    I.mu[s] = mu;
#pragma unroll
    for (int k = 0; k < 9; ++k) I.sig[k * N + s] = sig[k];
  }
}

// ---------------------------------------------------------------- staged path
// The antisymmetric part of the stress scratch, for the force of the form of Eqs. 9-11.
template <typename T, class NB = Nbr>
struct AntiSigAcc {
  const T* sg;
  long long N;
  NB nb;
  __device__ __forceinline__ T sig(int k, int cx, int cy, int cz) const {
    const int a = k / 3, b = k - 3 * a;
    if (a == b) return T(0);
    const long long o = nb.off(cx, cy, cz);
    return T(0.5) * (ld(sg + k * N + o) - ld(sg + (3 * b + a) * N + o));
  }
  // pair 4 holds sigma^A_zz = 0 (and no mu: the force does not read lane 1)
  __device__ __forceinline__ Vec2<T> spair(int j, int cx, int cy, int cz) const {
    if (j == 4) return Vec2<T>{T(0), T(0)};
    return Vec2<T>{sig(pair_c0(j), cx, cy, cz), sig(pair_c1(j), cx, cy, cz)};
  }
};

// k_lb: the force from the stress scratch, pull, moments and collision (a3, a5):
// g_out, u_out = velocity of this step.  FORM 0: F = div sigma, BGK + Guo (Eqs. 6-8).
// FORM 1: FA = div sigma^A and the equilibrium with sigma^S (Eqs. 9-11).
template <typename T, bool SHIFT, class V, int FORM, int ST>
__global__ void __launch_bounds__(kStepBlock) k_lb(const InstDesc<T>* __restrict__ D, int ninst) {
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
  auto nb = make_nbr_st<ST>(x, y, z, nx, ny, nz);
  using NB = decltype(nb);
  T F[3];
  if (FORM == 0) {
    GlobalAcc<T, NB> acc;
    acc.sg = I.sig;
    acc.N = N;
    acc.nb = nb;
    if constexpr (ST == 1) gather_force_r2<T>(acc, F);
    else gather_force<T>(acc, F);
  } else {
    AntiSigAcc<T, NB> acc{I.sig, N, nb};
    if constexpr (ST == 1) gather_force_r2<T>(acc, F);
    else gather_force<T>(acc, F);
  }
  T g[V::Q];
#pragma unroll
  for (int i = 0; i < V::Q; ++i) g[i] = ld(I.g_in + i * N + nb.off(-V::c(i, 0), -V::c(i, 1), -V::c(i, 2)));
  T u[3];
  if (FORM == 0) {
    lb_collide<T, SHIFT, V>(I.c, F, g, u);
  } else {
    T sg[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) sg[k] = I.sig[k * N + s];
    lb_collide_stress<T, SHIFT, V>(I.c, F, sg, g, u);
  }
#pragma unroll
  for (int i = 0; i < V::Q; ++i) I.g_out[i * N + s] = g[i];
#pragma unroll
  for (int a = 0; a < 3; ++a) I.u_out[a * N + s] = u[a];
}

// k_op: the order-parameter update (a4) of the staged path, advecting with u_in (lagged)
// or u_out (sync, written by k_lb of this step).
//   STAGE 0  Euler:           q_out = Q + R(Q)                        (H, mu from the scratch)
//   STAGE 1  Heun predictor:  rq = R(Q), qp = Q + rq
//   STAGE 2  Heun corrector:  q_out = Q + (rq + R(qp)) / 2            (H, mu of qp in sigma)
template <typename T, int STAGE, int ST>
__global__ void __launch_bounds__(kStepBlock) k_op(const InstDesc<T>* __restrict__ D, int ninst, int sync) {
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
  GlobalAcc<T, decltype(make_nbr_st<ST>(0, 0, 0, 4, 4, 4))> acc;
  acc.q_ = STAGE == 2 ? I.qp : I.q_in;
  acc.ps = STAGE == 2 ? I.qp + 5 * N : I.psi_in;
  acc.mu_ = STAGE == 2 ? I.sig + 5 * N : I.mu;
  acc.u_ = sync ? I.u_out : I.u_in;
  acc.N = N;
  acc.nb = make_nbr_st<ST>(x, y, z, nx, ny, nz);
  T lapmu, Wg[3][3], q0[5], qf[6][5], p0, pf[6], u0[3], uf[6];
  if constexpr (ST == 1) gather_op_r2<T>(acc, lapmu, Wg, q0, qf, p0, pf, u0, uf);
  else gather_op<T>(acc, lapmu, Wg, q0, qf, p0, pf, u0, uf);
  const T* Hsrc = STAGE == 2 ? I.sig : I.H;
  T Hs[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) Hs[k] = Hsrc[k * N + s];
  T qn[5], pn;
  if (STAGE == 0) {
    op_update<T, false>(I.c, lapmu, Wg, q0, qf, p0, pf, u0, uf, Hs, qn, pn);
#pragma unroll
    for (int k = 0; k < 5; ++k) I.q_out[k * N + s] = qn[k];
    I.psi_out[s] = pn;
  } else if (STAGE == 1) {
    op_update<T, true>(I.c, lapmu, Wg, q0, qf, p0, pf, u0, uf, Hs, qn, pn);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      I.rq[k * N + s] = qn[k];
      I.qp[k * N + s] = q0[k] + qn[k];
    }
    I.rq[5 * N + s] = pn;
    I.qp[5 * N + s] = p0 + pn;
  } else {
    op_update<T, true>(I.c, lapmu, Wg, q0, qf, p0, pf, u0, uf, Hs, qn, pn);
#pragma unroll
    for (int k = 0; k < 5; ++k) I.q_out[k * N + s] = I.q_in[k * N + s] + T(0.5) * (I.rq[k * N + s] + qn[k]);
    I.psi_out[s] = I.psi_in[s] + T(0.5) * (I.rq[5 * N + s] + pn);
  }
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
  GlobalAcc<T> acc;
  acc.q_ = I.q_in;
  acc.ps = I.psi_in;
  acc.sg = I.sig;
  acc.mu_ = I.mu;
  acc.u_ = I.u_in;
  acc.N = N;
  acc.nb = make_nbr(x, y, z, nx, ny, nz);
  T F[3], lapmu, Wg[3][3], q0[5], qf[6][5], p0, pf[6], u0[3], uf[6];
  gather_update<T>(acc, F, lapmu, Wg, q0, qf, p0, pf, u0, uf);
  T Hs[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) Hs[k] = I.H[k * N + s];
  T g[19];
#pragma unroll
  for (int i = 0; i < 19; ++i) g[i] = ld(I.g_in + i * N + acc.nb.off(-lat_c(i, 0), -lat_c(i, 1), -lat_c(i, 2)));
  T qn[5], pn, u[3];
  update_math<T, SHIFT>(I.c, F, lapmu, Wg, q0, qf, p0, pf, u0, uf, Hs, g, qn, pn, u);
#pragma unroll
  for (int k = 0; k < 5; ++k) I.q_out[k * N + s] = qn[k];
  I.psi_out[s] = pn;
#pragma unroll
  for (int i = 0; i < 19; ++i) I.g_out[i * N + s] = g[i];
#pragma unroll
  for (int a = 0; a < 3; ++a) I.u_out[a * N + s] = u[a];
}

// ---------------------------------------------------------------- field exchange
// dst components, in mask order: G(19) RHO(1) U(3) Q(5) PSI(1); offsets given per group
// (-1 = not selected).
template <typename T, bool SHIFT, class V>
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
      for (int i = 0; i < V::Q; ++i) {
        const long long src = nb.off(-V::c(i, 0), -V::c(i, 1), -V::c(i, 2));
        double fi = (double)I.g_in[i * N + src];
        if (SHIFT) fi += V::w(i) * (double)I.c.rho0;
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
template <typename T, bool SHIFT, class V>
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
      for (int i = 0; i < V::Q; ++i) {
        const long long d = nb.off(-V::c(i, 0), -V::c(i, 1), -V::c(i, 2));
        double fi = src[oG + i * N + s];
        if (SHIFT) fi -= V::w(i) * (double)I.c.rho0;
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
// a6 as a separate pass (state set from outside, or a path without the fused sums): FP64
// mass, sum psi, momentum (3), sum phi_c cos (3), sum phi_c sin (3) and sum phi_c of the
// populations stored at each site (streaming only permutes them, so the sums equal those of
// the pulled populations).  Each warp takes whole x rows (no index division per site); a lane
// adds its sites of a row in T, then into FP64; cos and sin come from the instance's tables.
// (s, c) += x, with s + x split by TwoSum (Knuth, TAOCP vol. 2, 4.2.2) into its rounded sum
// and its exact rounding error, which c gathers: s + c carries about twice T's precision.  The
// a6 sums of the FP32 path are formed this way, so they come out as the FP64 sums of the
// per-site FP32 shares.
// a * b rounded to T before any later use: the a6 shares are products that must come out as
// the same T values in every pass, so they may not be contracted into a following addition.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

template <typename T>
__device__ __forceinline__ void two_sum_add(T& s, T& c, T x) {
  const T t = s + x;
  const T bp = t - s;
  const T err = (s - (t - bp)) + (x - bp);
  s = t;
  c += err;
}

// k_obs_partial writes partial[block][12]; k_obs_final sums them in a fixed order.  Each
// thread adds the per-site shares (mass and momentum of the site's 19 stored populations, psi,
// phi_c and phi_c times the cos/sin tables, each formed in T as the fused step forms them) into
// error-free (sum, error) pairs, then FP64 takes over.
template <typename T, bool SHIFT, class V>
__global__ void __launch_bounds__(kObsBlock) k_obs_partial(InstDesc<T> I, double* __restrict__ partial) {
  T as[12], ac[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) as[k] = ac[k] = T(0);
  const int nx = I.nx, ny = I.ny;
  const long long N = I.N;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int WPB = kObsBlock / 32;
  const int rows = ny * I.nz;
  for (int r = blockIdx.x * WPB + wid; r < rows; r += gridDim.x * WPB) {
    const int y = r % ny, z = r / ny;
    const long long base = (long long)r * nx;
    const T cy = __ldg(I.trig + 2 * (nx + y)), sy = __ldg(I.trig + 2 * (nx + y) + 1);
    const T cz = __ldg(I.trig + 2 * (nx + ny + z)), sz = __ldg(I.trig + 2 * (nx + ny + z) + 1);
    for (int x = lane; x < nx; x += 32) {
      const long long st = base + x;
      T m = T(0), j0 = T(0), j1 = T(0), j2 = T(0);
#pragma unroll
      for (int i = 0; i < V::Q; ++i) {
        const T f = __ldg(I.g_in + i * N + st);
        m += f;
        if (V::c(i, 0)) j0 += V::c(i, 0) > 0 ? f : -f;
        if (V::c(i, 1)) j1 += V::c(i, 1) > 0 ? f : -f;
        if (V::c(i, 2)) j2 += V::c(i, 2) > 0 ? f : -f;
      }
      const T p = __ldg(I.psi_in + st);
      const T h = T(0.5) * (T(1) + p);
      const T v[12] = {m, p, j0, j1, j2, mul_rn(h, __ldg(I.trig + 2 * x)), mul_rn(h, cy), mul_rn(h, cz),
                       mul_rn(h, __ldg(I.trig + 2 * x + 1)), mul_rn(h, sy), mul_rn(h, sz), h};
#pragma unroll
      for (int k = 0; k < 12; ++k) two_sum_add(as[k], ac[k], v[k]);
    }
  }
  double acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = (double)as[k] + (double)ac[k];
  if (SHIFT && blockIdx.x == 0 && threadIdx.x == 0) acc[0] += (double)N * (double)I.c.rho0;
  __shared__ double sh[WPB][12];
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
    for (int w = 0; w < WPB; ++w) v += sh[w][threadIdx.x];
    partial[blockIdx.x * 12 + threadIdx.x] = v;
  }
}

// Sums partial[nblocks][12] into out[12]: thread (l, k) adds blocks l, l + 32, ... of value k,
// then the 32 subtotals of each value are added in order.
static __global__ void __launch_bounds__(384) k_obs_final(const double* __restrict__ partial, int nblocks,
                                                          double* __restrict__ out) {
  __shared__ double red[32][12];
  const int k = threadIdx.x % 12, l = threadIdx.x / 12;
  double v = 0.0;
  for (int b = l; b < nblocks; b += 32) v += partial[b * 12 + k];
  red[l][k] = v;
  __syncthreads();
  if (threadIdx.x < 12) {
    double t = 0.0;
    for (int q = 0; q < 32; ++q) t += red[q][threadIdx.x];
    out[threadIdx.x] = t;
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

template <typename T, bool SHIFT>
cudaError_t Launch<T, SHIFT>::fields(const InstDesc<T>* d_desc, int ninst, long long total_blocks, int bs,
                                     cudaStream_t s) {
  k_fields<T><<<(unsigned)total_blocks, bs, 0, s>>>(d_desc, ninst);
  return cudaGetLastError();
}

template <typename T, bool SHIFT, int ST>
cudaError_t staged_st(const InstDesc<T>* d_desc, int ninst, unsigned g, int bs, bool heun, bool sync, int vel,
                      int form, cudaStream_t s) {
  k_fields<T, false, ST><<<g, bs, 0, s>>>(d_desc, ninst);
  if (vel == 0 && form == 0) k_lb<T, SHIFT, VelD3Q19, 0, ST><<<g, bs, 0, s>>>(d_desc, ninst);
  else if (vel == 0) k_lb<T, SHIFT, VelD3Q19, 1, ST><<<g, bs, 0, s>>>(d_desc, ninst);
  else if (form == 0) k_lb<T, SHIFT, VelD3Q15, 0, ST><<<g, bs, 0, s>>>(d_desc, ninst);
  else k_lb<T, SHIFT, VelD3Q15, 1, ST><<<g, bs, 0, s>>>(d_desc, ninst);
  if (!heun) {
    k_op<T, 0, ST><<<g, bs, 0, s>>>(d_desc, ninst, sync ? 1 : 0);
  } else {
    k_op<T, 1, ST><<<g, bs, 0, s>>>(d_desc, ninst, sync ? 1 : 0);
    k_fields<T, true, ST><<<g, bs, 0, s>>>(d_desc, ninst);
    k_op<T, 2, ST><<<g, bs, 0, s>>>(d_desc, ninst, sync ? 1 : 0);
  }
  return cudaGetLastError();
}

template <typename T, bool SHIFT>
cudaError_t Launch<T, SHIFT>::staged(const InstDesc<T>* d_desc, int ninst, long long total_blocks, int bs, bool heun,
                                     bool sync, int vel, int form, int stencil, cudaStream_t s) {
  const unsigned g = (unsigned)total_blocks;
  if (stencil == 1) return staged_st<T, SHIFT, 1>(d_desc, ninst, g, bs, heun, sync, vel, form, s);
  return staged_st<T, SHIFT, 0>(d_desc, ninst, g, bs, heun, sync, vel, form, s);
}

inline unsigned grid_for(long long N, int bs) {
  long long g = (N + bs - 1) / bs;
  if (g > 152 * 16) g = 152 * 16;
  return (unsigned)(g < 1 ? 1 : g);
}

template <typename T, bool SHIFT>
cudaError_t Launch<T, SHIFT>::get_fields(const InstDesc<T>& I, uint32_t mask, double* dst, cudaStream_t s) {
  long long o = 0, oG = -1, oR = -1, oU = -1, oQ = -1, oP = -1;
  if (mask & 1u) { oG = o; o += (I.vel ? 15 : 19) * I.N; }
  if (mask & 2u) { oR = o; o += I.N; }
  if (mask & 4u) { oU = o; o += 3 * I.N; }
  if (mask & 8u) { oQ = o; o += 5 * I.N; }
  if (mask & 16u) { oP = o; o += I.N; }
  if (I.vel) k_get_fields<T, SHIFT, VelD3Q15><<<grid_for(I.N, 256), 256, 0, s>>>(I, oG, oR, oU, oQ, oP, dst);
  else k_get_fields<T, SHIFT, VelD3Q19><<<grid_for(I.N, 256), 256, 0, s>>>(I, oG, oR, oU, oQ, oP, dst);
  return cudaGetLastError();
}

template <typename T, bool SHIFT>
cudaError_t Launch<T, SHIFT>::set_fields(const InstDesc<T>& I, uint32_t mask, const double* src, T* g_t, T* q_t,
                                         T* p_t, T* u_t, cudaStream_t s) {
  long long o = 0, oG = -1, oU = -1, oQ = -1, oP = -1;
  if (mask & 1u) { oG = o; o += (I.vel ? 15 : 19) * I.N; }
  if (mask & 4u) { oU = o; o += 3 * I.N; }
  if (mask & 8u) { oQ = o; o += 5 * I.N; }
  if (mask & 16u) { oP = o; o += I.N; }
  if (I.vel)
    k_set_fields<T, SHIFT, VelD3Q15><<<grid_for(I.N, 256), 256, 0, s>>>(I, oG, oU, oQ, oP, src, g_t, q_t, p_t, u_t);
  else
    k_set_fields<T, SHIFT, VelD3Q19><<<grid_for(I.N, 256), 256, 0, s>>>(I, oG, oU, oQ, oP, src, g_t, q_t, p_t, u_t);
  return cudaGetLastError();
}

template <typename T, bool SHIFT>
cudaError_t Launch<T, SHIFT>::observables(const InstDesc<T>& I, double* partial, int nblocks, double* out,
                                          cudaStream_t s) {
  if (I.vel) k_obs_partial<T, SHIFT, VelD3Q15><<<nblocks, kObsBlock, 0, s>>>(I, partial);
  else k_obs_partial<T, SHIFT, VelD3Q19><<<nblocks, kObsBlock, 0, s>>>(I, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_obs_final<<<1, 384, 0, s>>>(partial, nblocks, out);
  return cudaGetLastError();
}

}  // namespace lbcad
