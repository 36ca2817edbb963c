// lbcad_fused.cuh -- the whole hybrid step in one persistent kernel.
//
// Each block owns a TX x TY column of the lattice and marches up z, keeping in shared
// memory rings of planes:
//   Q and psi with a halo of 2 (5 planes: z-1 .. z+3),
//   sigma (9) and mu with a halo of 1 (3 planes: z-1 .. z+1),
//   u of the previous step with a halo of 1 (4 planes: z-1 .. z+2),
// and the molecular field H of the next output plane in registers.  Per output plane z:
//   1. sigma phase: stencils, H, mu and sigma of plane z+1 on the tile plus a halo of 1
//      (the halo sites are the only redundant work: (TX+2)(TY+2)/(TX TY)).  The halo
//      sites take a second round on NHALO threads; the other threads meanwhile load the
//      Q/psi plane z+3 and the u plane z+2 for the next iteration;
//   2. output phase: F = div sigma, lap mu, grad u, upwind Q and psi, pull of the 19
//      populations from global memory, BGK + Guo collision; store g, Q, psi, u.
// Every global element of the state is read and written once per step by design (224 B per
// site in FP32); the halo re-reads of Q, psi and u and the x-shifted pulls come on top, as far
// as L2 does not hold them (tiles that neighbour in x run at different z).
//
// The grid is persistent: the flattened space of (tile column, z plane) work is split
// evenly across the blocks, so load balance does not depend on the box shape and one
// launch covers every instance of a batch.
//
// The end of the file holds the order-parameter half of the sync-coupled and Heun steps, as
// tiled z-marching kernels on the same tiles and work split.
#pragma once

#include <type_traits>

#include "lbcad_kernels.cuh"

namespace lbcad {

template <typename T, int TX, int TY>
struct FusedGeom {
  static constexpr int NT = TX * TY;
  static constexpr int QW = TX + 4, QH = TY + 4, QP = QW * QH;
  static constexpr int SW = TX + 2, SH = TY + 2, SP = SW * SH;
  static constexpr int QSLOT = 6 * QP, SSLOT = 10 * SP, USLOT = 3 * SP;
  // rings: Q/psi planes z-1 .. z+3, sigma/mu planes z-1 .. z+1, u planes z-1 .. z+2
  static constexpr int NQS = 5, NSS = 3, NUS = 4;
  static constexpr size_t elems = (size_t)NQS * QSLOT + (size_t)NSS * SSLOT + (size_t)NUS * USLOT;
  static constexpr int NW = NT / 32;  // warps adding to the a6 sums
  // a6 (kernels with the sums): per-warp accumulators [NW][12][2] in T, then the segment's 12
  // FP64 values
  static constexpr size_t obs_off = (elems * sizeof(T) + (QW + QH) * sizeof(int) + 15) / 16 * 16;
  static constexpr size_t seg_off = obs_off + (size_t)NW * 24 * sizeof(T);
  static constexpr size_t bytes_plain = elems * sizeof(T) + (QW + QH) * sizeof(int);
  static constexpr size_t bytes_obs = seg_off + 12 * sizeof(double);
  static constexpr size_t bytes(bool obs) { return obs ? bytes_obs : bytes_plain; }
  static constexpr int NHALO = SP - NT;   // halo sites of the sigma phase (second round)
  static constexpr int NLOAD = NT - NHALO;  // threads free to prefetch during that round
  static_assert(NHALO > 0 && NHALO < NT, "halo sites must fit in one extra round");
  static constexpr int QLD = (QP + NLOAD - 1) / NLOAD;  // Q sites each loader thread fetches
  static constexpr int ULD = (SP + NLOAD - 1) / NLOAD;
};

// Periodic plane index for p in [-n, 2n): the planes a column segment touches lie in
// [-2, nz + 3] and every edge is >= 4, so one add or subtract suffices (no division).
__device__ __forceinline__ int wrap_plane(int p, int n) { return p < 0 ? p + n : (p >= n ? p - n : p); }

__device__ __forceinline__ int wrapmod(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// Shared-memory Q/psi plane: the six fields in interleaved pairs (Q_xx, Q_xy), (Q_xz, Q_yy),
// (Q_yz, psi); field f of tile site k sits at element (f >> 1) * 2 QP + 2 k + (f & 1), so a
// pair is one aligned two-element load.
template <int QP>
__device__ __forceinline__ int qidx(int f, int k) {
  return (f >> 1) * 2 * QP + 2 * k + (f & 1);
}

template <typename T, int QW, int QP>
struct SmemFieldsAcc {
  const T* pl[3];  // Q/psi planes p-1, p, p+1
  int qc;          // tile index of the centre site
  __device__ __forceinline__ T q(int k, int cx, int cy, int cz) const {
    return pl[cz + 1][qidx<QP>(k, qc + cy * QW + cx)];
  }
  __device__ __forceinline__ T psi(int cx, int cy, int cz) const { return pl[cz + 1][qidx<QP>(5, qc + cy * QW + cx)]; }
  __device__ __forceinline__ Vec2<T> pair(int j, int cx, int cy, int cz) const {
    const T* p = pl[cz + 1] + qidx<QP>(2 * j, qc + cy * QW + cx);
    if constexpr (sizeof(T) == 4) {
      const float2 v = *reinterpret_cast<const float2*>(p);
      return Vec2<T>{v.x, v.y};
    } else {
      const double2 v = *reinterpret_cast<const double2*>(p);
      return Vec2<T>{v.x, v.y};
    }
  }
};

// Shared-memory sigma/mu plane: five pairs (see sig_pair), pair j of tile site k at
// elements j * 2 SP + 2 k (+1).  Velocity plane: (u_x, u_y) of site k at 2 k (+1), u_z at
// 2 SP + k.
template <int SP>
__device__ __forceinline__ int uidx(int a, int k) {
  return a < 2 ? 2 * k + a : 2 * SP + k;
}

template <typename T>
__device__ __forceinline__ Vec2<T> lds2(const T* p) {
  if constexpr (sizeof(T) == 4) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    return Vec2<T>{v.x, v.y};
  } else {
    const double2 v = *reinterpret_cast<const double2*>(p);
    return Vec2<T>{v.x, v.y};
  }
}

// An aligned pair from global memory through the read-only path.
template <typename T>
__device__ __forceinline__ Vec2<T> ldg2(const T* p) {
  if constexpr (sizeof(T) == 4) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return Vec2<T>{v.x, v.y};
  } else {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    return Vec2<T>{v.x, v.y};
  }
}

template <typename T, int QW, int QP, int SW, int SP>
struct SmemUpdateAcc {
  const T* qpl[3];
  const T* spl[3];
  const T* upl[3];
  int qc;  // tile index of the centre site in the Q/psi plane
  int sc;  // ... in the sigma and u planes
  __device__ __forceinline__ T q(int k, int cx, int cy, int cz) const {
    return qpl[cz + 1][qidx<QP>(k, qc + cy * QW + cx)];
  }
  __device__ __forceinline__ T psi(int cx, int cy, int cz) const { return qpl[cz + 1][qidx<QP>(5, qc + cy * QW + cx)]; }
  __device__ __forceinline__ Vec2<T> pair(int j, int cx, int cy, int cz) const {
    return lds2(qpl[cz + 1] + qidx<QP>(2 * j, qc + cy * QW + cx));
  }
  __device__ __forceinline__ Vec2<T> spair(int j, int cx, int cy, int cz) const {
    return lds2(spl[cz + 1] + j * 2 * SP + 2 * (sc + cy * SW + cx));
  }
  __device__ __forceinline__ Vec2<T> upair(int cx, int cy, int cz) const {
    return lds2(upl[cz + 1] + 2 * (sc + cy * SW + cx));
  }
  __device__ __forceinline__ T u(int a, int cx, int cy, int cz) const {
    return upl[cz + 1][uidx<SP>(a, sc + cy * SW + cx)];
  }
};

// The stress and mu of tile site k into a sigma plane as five pairs (two-element stores).
template <typename T, int SP>
__device__ __forceinline__ void store_sigma(T* plane, int k, const T sig[9], T mu) {
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    T* p = plane + j * 2 * SP + 2 * k;
    const T a = sig[pair_c0(j)], b = j == 4 ? mu : sig[pair_c1(j)];
    if constexpr (sizeof(T) == 4) *reinterpret_cast<float2*>(p) = make_float2(a, b);
    else *reinterpret_cast<double2*>(p) = make_double2(a, b);
  }
}

// Component c (= 3a + b) of the stress at an offset, through an accessor of stress pairs.
template <typename T, class A>
__device__ __forceinline__ T pair_comp(const A& acc, int c, int cx, int cy, int cz) {
  const Vec2<T> v = acc.spair(sig_pair(c), cx, cy, cz);
  return sig_lane(c) ? v.y : v.x;
}

// The antisymmetric part sigma^A = (sigma - sigma^T)/2 through an accessor of stress pairs
// (the force of the Eq. 9-11 form); pair 4 holds sigma^A_zz = 0 and no mu.
template <typename T, class A>
struct AntiPairAcc {
  A a;
  __device__ __forceinline__ T anti(int c, int cx, int cy, int cz) const {
    const int r = c / 3, k = c - 3 * r;
    if (r == k) return T(0);
    return T(0.5) * (pair_comp<T>(a, c, cx, cy, cz) - pair_comp<T>(a, 3 * k + r, cx, cy, cz));
  }
  __device__ __forceinline__ Vec2<T> spair(int j, int cx, int cy, int cz) const {
    if (j == 4) return Vec2<T>{T(0), T(0)};
    return Vec2<T>{anti(pair_c0(j), cx, cy, cz), anti(pair_c1(j), cx, cy, cz)};
  }
};

// The output work of one site (a3 - a5) from the shared-memory tiles: the force, the
// stencils of a4, the pull of the populations of velocity set V, the order-parameter update
// and the collision; stores g, Q, psi and u.  FORM 0: F = div sigma, BGK + Guo (Eqs. 6-8).
// FORM 1: FA = div sigma^A and the equilibrium carrying sigma^S (Eqs. 9-11).
// offs(zo, pyo, pxo) fills the global offsets of the planes z-1, z, z+1, the rows y-1, y, y+1
// and the columns x-1, x, x+1, and hs(H) the molecular field of the site; both are called
// late (after the stencils, after the pulls), so that their values do not hold registers
// through the earlier work.  pull(g, zo, pyo, pxo) fills the pulled populations g_i(x - c_i)
// (GlobalPull: from global memory at those offsets).  ob (OBS): the site's share of the a6
// sums of the new state (see FusedObs); trg(tx, ty, tz) gives (cos, sin) of 2 pi x/nx,
// 2 pi y/ny and 2 pi z/nz of the site.
// The pulls address population i of plane z - c_z through a base pointer that is the same for
// the whole block (g_in + i N + plane offset) plus the site's in-plane offset of row y - c_y and
// column x - c_x (below 2^31, so 32-bit): one 64-bit addition per pull.
template <typename T, class V>
struct GlobalPull {
  const T* g_in;
  long long N;
  __device__ __forceinline__ void operator()(T g[V::Q], const long long zo[3], const int pyo[3],
                                             const int pxo[3]) const {
#pragma unroll
    for (int i = 0; i < V::Q; ++i) {
      const T* base = g_in + (i * N + zo[1 - V::c(i, 2)]);
      const unsigned o = (unsigned)(pyo[1 - V::c(i, 1)] + pxo[1 - V::c(i, 0)]);
      g[i] = ld(base + o);
    }
  }
};

// A store of an output value to global memory, cached in L2 only: the next step reads the new
// state back through L2, and the pulls of this step keep L1 to themselves.
template <typename T>
__device__ __forceinline__ void st_out(T* p, T v) {
  __stcg(p, v);
}

template <typename T, bool SHIFT, class V, int FORM, int MODE, class A, class Offs, class HS, class TR, class PL>
__device__ __forceinline__ void output_site(const InstDesc<T>& I, const Coef<T>& cf, const A& acc, const Offs& offs,
                                            const HS& hs, const TR& trg, const PL& pull, T ob[12]) {
  constexpr bool OBS = MODE == kFusedSums;
  const long long N = I.N;
  if constexpr (MODE == kFusedLbOnly) {
    // sync coupling, first half: force, pull and collision (u of this step), and H and mu of
    // the site into the scratch that the order-parameter kernel reads
    T F[3];
    if constexpr (FORM == 0) gather_force<T>(acc, F);
    else gather_force<T>(AntiPairAcc<T, A>{acc}, F);
    long long zo[3];
    int pyo[3], pxo[3];
    offs(zo, pyo, pxo);
    T g[V::Q];
    pull(g, zo, pyo, pxo);
    T u[3];
    if constexpr (FORM == 0) {
      lb_collide<T, SHIFT, V>(cf, F, g, u);
    } else {
      T sg[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) sg[c] = pair_comp<T>(acc, c, 0, 0, 0);
      lb_collide_stress<T, SHIFT, V>(cf, F, sg, g, u);
    }
    const long long s = zo[1] + pyo[1] + pxo[1];
    T* const go = I.g_out + s;
    T* const uo = I.u_out + s;
#pragma unroll
    for (int i = 0; i < V::Q; ++i) st_out(go + i * N, g[i]);
#pragma unroll
    for (int a = 0; a < 3; ++a) st_out(uo + a * N, u[a]);
    T Hs[5];
    hs(Hs);
    T* const ho = I.H + s;
#pragma unroll
    for (int k = 0; k < 5; ++k) st_out(ho + k * N, Hs[k]);
    st_out(I.mu + s, acc.spair(4, 0, 0, 0).y);
    return;
  }
  T F[3], lapmu, Wg[3][3], q0[5], qf[6][5], p0, pf[6], u0[3], uf[6];
  if constexpr (FORM == 0) gather_force<T>(acc, F);
  else gather_force<T>(AntiPairAcc<T, A>{acc}, F);
  gather_op<T>(acc, lapmu, Wg, q0, qf, p0, pf, u0, uf);
  long long zo[3];
  int pyo[3], pxo[3];
  offs(zo, pyo, pxo);
  T g[V::Q];
  pull(g, zo, pyo, pxo);
  T Hs[5], qn[5], pn, u[3], mom[4];
  hs(Hs);
  op_update<T, false>(cf, lapmu, Wg, q0, qf, p0, pf, u0, uf, Hs, qn, pn);
  if constexpr (FORM == 0) {
    lb_collide<T, SHIFT, V>(cf, F, g, u, OBS ? mom : nullptr);
  } else {
    T sg[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) sg[c] = pair_comp<T>(acc, c, 0, 0, 0);
    lb_collide_stress<T, SHIFT, V>(cf, F, sg, g, u, OBS ? mom : nullptr);
  }
  const long long s = zo[1] + pyo[1] + pxo[1];
  T* const qo = I.q_out + s;
  T* const go = I.g_out + s;
  T* const uo = I.u_out + s;
#pragma unroll
  for (int k = 0; k < 5; ++k) st_out(qo + k * N, qn[k]);
  st_out(I.psi_out + s, pn);
#pragma unroll
  for (int i = 0; i < V::Q; ++i) st_out(go + i * N, g[i]);
#pragma unroll
  for (int a = 0; a < 3; ++a) st_out(uo + a * N, u[a]);
  // a6: mass, psi and momentum of the new state, and phi_c with its centroid moments
  if constexpr (OBS) {
    const T pc = T(0.5) * (T(1) + pn);
    ob[0] = mom[0];
    ob[1] = pn;
    ob[2] = mom[1];
    ob[3] = mom[2];
    ob[4] = mom[3];
    ob[11] = pc;
    Vec2<T> tx, ty, tz;
    trg(tx, ty, tz);
    ob[5] = mul_rn(pc, tx.x);
    ob[6] = mul_rn(pc, ty.x);
    ob[7] = mul_rn(pc, tz.x);
    ob[8] = mul_rn(pc, tx.y);
    ob[9] = mul_rn(pc, ty.y);
    ob[10] = mul_rn(pc, tz.y);
  }
}

// The a6 sums within a block.  Per plane they are added in the compute type T: FP64
// arithmetic is slow on this part, and a few FP64 operations per plane on the critical path of
// the step cost a third of its speed.  The additions are error-free instead (two_sum_add):
// every sum is kept as an unevaluated pair (s, c) whose exact value is s + c, each addition
// split into its rounded result and its exact rounding error, the errors gathered in c.  The pair carries about twice T's precision (the only loss is the
// rounding of c itself, second order in T's unit roundoff), and FP64 takes over at the end of
// each column segment as (double)s + (double)c.  So the sums of the FP32 state come out as its
// FP64 sums, up to the FP32 rounding of each site's own share.

// Butterfly sum of the twelve values across the warp as (sum, error) pairs (every lane receives
// the pair of the warp), then lane k < 12 adds pair k to the warp's accumulator acc_w[k] =
// (sum, error).  FP64 values take a plain butterfly.
template <typename T>
__device__ __forceinline__ void obs_warp_add(T v[12], T* acc_w) {
  if constexpr (sizeof(T) == 8) {
    // FP64 values: a plain butterfly already carries the sums to FP64 rounding
#pragma unroll
    for (int k = 0; k < 12; ++k) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    }
    const int lane = threadIdx.x & 31;
    T mine = T(0);
#pragma unroll
    for (int k = 0; k < 12; ++k) mine = lane == k ? v[k] : mine;
    if (lane < 12) {
      T* a = acc_w + 2 * lane;
      T s = a[0], c = a[1];
      two_sum_add(s, c, mine);
      a[0] = s;
      a[1] = c;
    }
    return;
  }
  T e[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    e[k] = T(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T vo = __shfl_xor_sync(0xffffffffu, v[k], o);
      const T eo = __shfl_xor_sync(0xffffffffu, e[k], o);
      two_sum_add(v[k], e[k], vo);
      e[k] += eo;
    }
  }
  const int lane = threadIdx.x & 31;
  T mine = T(0), mine_e = T(0);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    mine = lane == k ? v[k] : mine;
    mine_e = lane == k ? e[k] : mine_e;
  }
  if (lane < 12) {
    T* a = acc_w + 2 * lane;
    T s = a[0], c = a[1];
    two_sum_add(s, c, mine);
    a[0] = s;
    a[1] = c + mine_e;
  }
}


// red[k + 12 m] (k < 12, m < M) summed over m into red[k] by a fixed pairing tree (all threads;
// barriers between the levels).  FP64 additions are long-latency on this part, so the sums run
// as trees of depth log2(M) rather than as chains of length M; the order is fixed, so the
// result does not depend on timing.
__device__ __forceinline__ void obs_tree12(double* red, int M) {
  for (int len = M; len > 1;) {
    const int half = (len + 1) >> 1;
    for (int t = threadIdx.x; t < 12 * (len - half); t += blockDim.x) red[t] += red[t + 12 * half];
    __syncthreads();
    len = half;
  }
}

// End of a column segment: its twelve FP64 sums go to the segment's slot with plain stores
// (threads 0-11, after a barrier that made seg[12] visible).  Nothing else happens per segment:
// the completion of an instance is counted once per block, at the end of the kernel
// (obs_block_end).
__device__ __forceinline__ void obs_segment_write(const FusedObs& ob, int slot, const double* seg) {
  if (threadIdx.x < 12) ob.slots[slot * 12 + threadIdx.x] = seg[threadIdx.x];
}

// End of the kernel (all threads): each segment of this block counts its slot on the
// segment's instance (after one fence for all of this block's slot stores); the block whose
// count completes an instance sums that instance's slots into ob.latest: each of the twelve
// values over fixed strided subsets of the slots, the loads of a thread in flight together,
// then over the subsets in order, so the result does not depend on which block finishes last.
// No spin waits.  red: shared scratch of at least 12 * (blockDim.x / 12) doubles.
// mass_shift(inst) = N rho0 with shifted populations, else 0.
template <class MS>
__device__ __forceinline__ void obs_block_end(const FusedObs& ob, int nseg, double* red, const MS& mass_shift) {
  __shared__ int last;
  const int tid = threadIdx.x;
  __syncthreads();
  if (tid < 12) __threadfence();  // the slot stores of this block's segments, before the counting
  __syncthreads();
  for (int j = 0; j < nseg; ++j) {
    const int inst = ob.slot_inst[blockIdx.x * ob.maxseg + j];
    if (tid == 0) last = atomicAdd(&ob.cnt[inst], 1u) == (unsigned)(ob.nslot[inst] - 1);
    __syncthreads();
    if (last) {
      __threadfence();
      const int per = blockDim.x / 12;
      const int lo = ob.slot_lo[inst], hi = ob.slot_hi[inst];
      if (tid < 12 * per) {
        const int k = tid % 12, l = tid / 12;
        double v = 0.0;
#pragma unroll 8
        for (int sl = lo + l; sl < hi; sl += per) {
          const int si = __ldg(ob.slot_inst + sl);
          const double x = __ldcg(ob.slots + sl * 12 + k);
          v += si == inst ? x : 0.0;
        }
        red[l * 12 + k] = v;
      }
      __syncthreads();
      obs_tree12(red, per);
      if (tid < 12) ob.latest[inst * 12 + tid] = red[tid] + (tid == 0 ? mass_shift(inst) : 0.0);
      if (tid == 0) ob.cnt[inst] = 0u;
    }
    __syncthreads();
  }
}

// Pipelined kernel: the a6 shares of an output plane (sh[IP][12], site-major, left in shared
// memory by the output warps) are added up in the next phase by the sigma threads that have no
// site in the last sigma round, while the others finish it: threads R0 .. R0 + NR - 1 (G::R0,
// G::NR, NR a multiple of 12).  Thread t = tid - R0 adds the elements t, t + NR, t + 2 NR, ...
// (all of value t % 12, consecutive addresses across a warp) into its own error-free pair
// acc[t] = (sum, error): no shuffles and no atomics.  (A two-lane form, two values per thread
// and f32x2 operations, measured slower: its dependency chains got no shorter.)
template <typename T, class G>
__device__ __forceinline__ void obs_sigma_reduce(const T* sh, T* acc) {
  const int t = (int)threadIdx.x - G::R0;
  if (t < 0 || t >= G::NR) return;
  T s = acc[2 * t], c = acc[2 * t + 1];
#pragma unroll 4
  for (int e = t; e < 12 * G::IP; e += G::NR) two_sum_add(s, c, sh[e]);
  acc[2 * t] = s;
  acc[2 * t + 1] = c;
}

// The twelve FP64 values of a pipelined segment from the sigma threads' accumulators: every
// accumulator converted in parallel into dred[NR] (shared scratch), then value k added over its
// threads t = k, k + 12, ... by a fixed tree.  All threads; seg[0..11] (threads 0-11) is visible
// after the caller's next barrier.
template <typename T, class G>
__device__ __forceinline__ void obs_sigma_values(const T* acc, double* dred, double* seg) {
  const int t = (int)threadIdx.x - G::R0;
  if (t >= 0 && t < G::NR) dred[t] = (double)acc[2 * t] + (double)acc[2 * t + 1];
  __syncthreads();
  obs_tree12(dred, G::NR / 12);
  if (threadIdx.x < 12) seg[threadIdx.x] = dred[threadIdx.x];
}

// Ring slots of plane p (p >= -2).
__device__ __forceinline__ int qslot(int p) { return (p + 10) % 5; }
__device__ __forceinline__ int sslot(int p) { return (p + 9) % 3; }
__device__ __forceinline__ int uslot(int p) { return (p + 8) % 4; }

template <typename T, bool SHIFT, int TX, int TY, class V, int FORM, int MODE>
__global__ void __launch_bounds__(TX * TY, (sizeof(T) == 4 && TX * TY <= 256) ? 2 : 1)
    k_step_fused(const InstDesc<T>* __restrict__ D, const FusedTile* __restrict__ tiles, int ntiles,
                 long long total, FusedObs ob) {
  constexpr bool OBS = MODE == kFusedSums;
  using G = FusedGeom<T, TX, TY>;
  constexpr int QW = G::QW, QP = G::QP, SW = G::SW, SH = G::SH, SP = G::SP, NT = G::NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sQ = reinterpret_cast<T*>(smem_raw);
  T* sS = sQ + G::NQS * G::QSLOT;
  T* sU = sS + G::NSS * G::SSLOT;
  int* xmap = reinterpret_cast<int*>(sU + G::NUS * G::USLOT);  // global x of Q-tile column
  int* ymap = xmap + QW;                                         // global y * nx of Q-tile row
  T* oacc = reinterpret_cast<T*>(smem_raw + G::obs_off);                 // a6 sums per warp [NW][12][2]
  double* oseg = reinterpret_cast<double*>(smem_raw + G::seg_off);       // a6 sums of the segment [12]
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;

  // this thread's halo site of the sigma phase (threads < NHALO)
  int hx = 0, hy = 0;
  if (tid < G::NHALO) {
    if (tid < 2 * SW) {
      hy = tid < SW ? 0 : SH - 1;
      hx = tid < SW ? tid : tid - SW;
    } else {
      const int r = tid - 2 * SW;
      hy = 1 + (r >> 1);
      hx = (r & 1) ? SW - 1 : 0;
    }
  }
  const int lt = tid - G::NHALO;  // loader index (threads >= NHALO)

  const long long begin = (total * blockIdx.x) / gridDim.x;
  const long long end = (total * (blockIdx.x + 1)) / gridDim.x;
  long long it = begin;
  int seg = 0;  // ordinal of the column segment within this block (its a6 slot)
  while (it < end) {
    int lo = 0, hi = ntiles - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tiles[mid].start <= it) lo = mid; else hi = mid - 1;
    }
    const FusedTile tl = tiles[lo];
    const InstDesc<T>& I = D[tl.inst];
    const int nx = I.nx, ny = I.ny, nz = I.nz;
    const long long N = I.N;
    const long long plane = (long long)nx * ny;
    const int zb = (int)(it - tl.start);
    const long long seg_end = end < tl.start + tl.nz ? end : tl.start + tl.nz;
    const int ze = (int)(seg_end - tl.start);
    it = seg_end;
    const Coef<T> cf = I.c;
    const T* __restrict__ qin = I.q_in;
    const T* __restrict__ pin = I.psi_in;
    const T* __restrict__ uin = I.u_in;

    __syncthreads();  // the previous segment is done with the shared tiles
    for (int k = tid; k < QW; k += NT) xmap[k] = wrapmod(tl.x0 + k - 2, nx);
    for (int k = tid; k < G::QH; k += NT) ymap[k] = wrapmod(tl.y0 + k - 2, ny) * nx;
    if constexpr (OBS)
      for (int k = tid; k < G::NW * 24; k += NT) oacc[k] = T(0);
    __syncthreads();

    // planes are loaded by a fixed set of tile positions per thread: their in-plane
    // global offsets are computed once per segment
    auto load_q_all = [&](int p) {  // every thread (prologue)
      T* dst = sQ + qslot(p) * G::QSLOT;
      const long long gz = (long long)wrap_plane(p, nz) * plane;
      for (int k = tid; k < QP; k += NT) {
        const int ly = k / QW, lx = k - ly * QW;
        const long long gs = gz + ymap[ly] + xmap[lx];
#pragma unroll
        for (int f = 0; f < 5; ++f) dst[qidx<QP>(f, k)] = ld(qin + f * N + gs);
        dst[qidx<QP>(5, k)] = ld(pin + gs);
      }
    };
    auto load_u_all = [&](int p) {
      T* dst = sU + uslot(p) * G::USLOT;
      const long long gz = (long long)wrap_plane(p, nz) * plane;
      for (int k = tid; k < SP; k += NT) {
        const int sy = k / SW, sx = k - sy * SW;
        const long long gs = gz + ymap[sy + 1] + xmap[sx + 1];
#pragma unroll
        for (int a = 0; a < 3; ++a) dst[uidx<SP>(a, k)] = ld(uin + a * N + gs);
      }
    };
    int qoff[G::QLD], uoff[G::ULD];
    if (lt >= 0) {
#pragma unroll
      for (int j = 0; j < G::QLD; ++j) {
        const int k = lt + j * G::NLOAD;
        if (k < QP) {
          const int ly = k / QW, lx = k - ly * QW;
          qoff[j] = ymap[ly] + xmap[lx];
        }
      }
#pragma unroll
      for (int j = 0; j < G::ULD; ++j) {
        const int k = lt + j * G::NLOAD;
        if (k < SP) {
          const int sy = k / SW, sx = k - sy * SW;
          uoff[j] = ymap[sy + 1] + xmap[sx + 1];
        }
      }
    }
    // prefetch by the loader threads: Q/psi plane pq and u plane pu
    auto prefetch = [&](int pq, int pu) {
      T* dq = sQ + qslot(pq) * G::QSLOT;
      const long long gzq = (long long)wrap_plane(pq, nz) * plane;
#pragma unroll
      for (int j = 0; j < G::QLD; ++j) {
        const int k = lt + j * G::NLOAD;
        if (k < QP) {
          const long long gs = gzq + qoff[j];
#pragma unroll
          for (int f = 0; f < 5; ++f) dq[qidx<QP>(f, k)] = ld(qin + f * N + gs);
          dq[qidx<QP>(5, k)] = ld(pin + gs);
        }
      }
      if constexpr (MODE == kFusedLbOnly) return;  // the LB half reads no previous u
      T* du = sU + uslot(pu) * G::USLOT;
      const long long gzu = (long long)wrap_plane(pu, nz) * plane;
#pragma unroll
      for (int j = 0; j < G::ULD; ++j) {
        const int k = lt + j * G::NLOAD;
        if (k < SP) {
          const long long gs = gzu + uoff[j];
#pragma unroll
          for (int a = 0; a < 3; ++a) du[uidx<SP>(a, k)] = ld(uin + a * N + gs);
        }
      }
    };
    // H, mu and sigma of plane p at sigma-tile site (sx, sy); returns H.
    auto sigma_site = [&](int p, int sx, int sy, T H[5]) {
      SmemFieldsAcc<T, QW, QP> acc;
      acc.qc = (sy + 1) * QW + (sx + 1);
#pragma unroll
      for (int j = 0; j < 3; ++j) acc.pl[j] = sQ + qslot(p - 1 + j) * G::QSLOT;
      T q0[5], p0, dq[3][5], lapq[5], dp[3], lapp, hp[6];
      gather_fields<T>(acc, q0, p0, dq, lapq, dp, lapp, hp);
      T sig[9], mu;
      local_fields<T>(cf, q0, p0, dq, lapq, dp, lapp, hp, H, mu, sig);
      store_sigma<T, SP>(sS + sslot(p) * G::SSLOT, sy * SW + sx, sig, mu);
    };

    load_q_all(zb - 2);
    load_q_all(zb - 1);
    load_q_all(zb);
    if constexpr (MODE != kFusedLbOnly) load_u_all(zb - 1);  // the LB half reads no previous u
    T Hc[5] = {T(0), T(0), T(0), T(0), T(0)};
    for (int z = zb - 2; z < ze; ++z) {
      __syncthreads();  // Q(z .. z+2) and u(z-1 .. z+1) resident; the previous output phase is done
      // sigma phase for plane z+1: interior sites first (their H is kept for the next
      // output plane), then the halo sites while the other threads prefetch
      // Q(z+3) and u(z+2) into the slots of Q(z-2) and u(z-2)
      T Hn[5];
#pragma unroll 1
      for (int r = 0; r < 2; ++r) {  // one copy of the sigma code for both rounds
        if (r == 1 && tid >= G::NHALO) break;
        const int sx = r ? hx : tx + 1, sy = r ? hy : ty + 1;
        T H[5];
        sigma_site(z + 1, sx, sy, H);
        if (r == 0) {
#pragma unroll
          for (int k = 0; k < 5; ++k) Hn[k] = H[k];
        }
      }
      if (tid >= G::NHALO) prefetch(z + 3, z + 2);
      __syncthreads();
      T ob6[12] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
      if (z >= zb && tl.x0 + tx < nx && tl.y0 + ty < ny) {
        SmemUpdateAcc<T, QW, QP, SW, SP> acc;
        acc.qc = (ty + 2) * QW + (tx + 2);
        acc.sc = (ty + 1) * SW + (tx + 1);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          acc.qpl[j] = sQ + qslot(z - 1 + j) * G::QSLOT;
          acc.spl[j] = sS + sslot(z - 1 + j) * G::SSLOT;
          acc.upl[j] = sU + uslot(z - 1 + j) * G::USLOT;
        }
        // offsets of this thread's output site and its neighbours (pull)
        auto offs = [&](long long zo[3], int pyo[3], int pxo[3]) {
          zo[0] = (long long)wrap_plane(z - 1, nz) * plane;
          zo[1] = (long long)z * plane;
          zo[2] = (long long)wrap_plane(z + 1, nz) * plane;
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            pyo[j] = ymap[ty + 1 + j];
            pxo[j] = xmap[tx + 1 + j];
          }
        };
        auto hs = [&](T H[5]) {
#pragma unroll
          for (int c = 0; c < 5; ++c) H[c] = Hc[c];
        };
        auto trg = [&](Vec2<T>& ctx, Vec2<T>& cty, Vec2<T>& ctz) {
          ctx = ldg2(I.trig + 2 * (tl.x0 + tx));
          cty = ldg2(I.trig + 2 * (nx + tl.y0 + ty));
          ctz = ldg2(I.trig + 2 * (nx + ny + z));
        };
        output_site<T, SHIFT, V, FORM, MODE>(I, cf, acc, offs, hs, trg, GlobalPull<T, V>{I.g_in, N}, ob6);
      }
      if constexpr (OBS)
        if (z >= zb) obs_warp_add<T>(ob6, oacc + (tid >> 5) * 24);
#pragma unroll
      for (int k = 0; k < 5; ++k) Hc[k] = Hn[k];
    }
    if constexpr (OBS) {
      __syncthreads();
      double* dred = reinterpret_cast<double*>(smem_raw);
      if (tid < 12 * G::NW) dred[tid] = (double)oacc[2 * tid] + (double)oacc[2 * tid + 1];
      __syncthreads();
      obs_tree12(dred, G::NW);
      if (tid < 12) oseg[tid] = dred[tid];
      __syncthreads();
      obs_segment_write(ob, blockIdx.x * ob.maxseg + seg, oseg);
    }
    ++seg;
  }
  if constexpr (OBS)
    obs_block_end(ob, seg, reinterpret_cast<double*>(smem_raw),
                  [&](int inst) { return SHIFT ? (double)D[inst].c.rho0 * (double)D[inst].N : 0.0; });
}

// ---------------------------------------------------------------- pipelined variant
// Same per-site arithmetic, different schedule: 32xTY tiles, 16 warps.  The first NS
// threads compute sigma, mu and H of plane k+1 (the 34 x (TY+2) sigma-tile sites, in
// rounds when NS is smaller) while the other 512 - NS threads compute the output of
// plane k-1 (one site each), in the same phase; one barrier per plane.  With TY = 6 both
// groups finish their plane in a single round (272 sigma sites, 192 outputs).  The output half carries the population pulls
// and the stores, so memory traffic overlaps the sigma arithmetic.  Planes for the next
// phase arrive by cp.async during the phase.
// Rings: Q/psi 6 planes (k-2 .. k+3), sigma/mu 4 (k-2 .. k+1), H 3 (k-1 .. k+1),
// u 4 (k-2 .. k+1).
template <int TY_, int NS_>
struct PipeGeom {
  static constexpr int TX = 32, TY = TY_, NT = 512, NS = NS_, NO = NT - NS;
  static constexpr int QW = TX + 4, QH = TY + 4, QP = QW * QH;
  static constexpr int SW = TX + 2, SH = TY + 2, SP = SW * SH;
  static constexpr int IP = TX * TY;
  static constexpr int NQS = 6, NSS = 4, NHS = 3, NUS = 4;
  static_assert(QP <= NT && SP <= NT && SP <= 2 * NS && NO >= IP, "site counts per thread");
  static_assert(NS % 32 == 0, "whole warps per group");
  // a6 reducers: the sigma threads from R0 on, which have no site in the last sigma round
  // (R0 rounded up to a warp where that leaves at least 12 threads)
  static constexpr int RL = SP - (SP - 1) / NS * NS;  // sites of the last sigma round
  static constexpr int R0 = ((RL + 31) / 32 * 32 < NS - 12) ? (RL + 31) / 32 * 32 : NS - 12;
  static constexpr int NR = (NS - R0) / 12 * 12;
  static_assert(NR >= 12, "a6 reducer threads");
  // a6: the output planes' shares [2][IP][12] (double-buffered by plane parity), the sigma
  // threads' accumulators [NR][2] in T, the tile's (cos, sin) of x and y [TX + TY][2], then
  // the segment's 12 FP64 values
  template <typename T>
  __host__ __device__ static constexpr size_t obs_off() {
    return (((size_t)NQS * 6 * QP + (size_t)NSS * 10 * SP + (size_t)NHS * 5 * IP + (size_t)NUS * 3 * SP) * sizeof(T) +
            (QW + QH) * sizeof(int) + 15) / 16 * 16;
  }
  template <typename T>
  __host__ __device__ static constexpr size_t acc_off() {
    return obs_off<T>() + (size_t)2 * IP * 12 * sizeof(T);
  }
  template <typename T>
  __host__ __device__ static constexpr size_t trig_off() {
    return acc_off<T>() + (size_t)NR * 2 * sizeof(T);
  }
  template <typename T>
  __host__ __device__ static constexpr size_t seg_off() {
    return (trig_off<T>() + (size_t)(TX + TY) * 2 * sizeof(T) + 7) / 8 * 8;
  }
  template <typename T>
  __host__ __device__ static constexpr size_t bytes(bool obs) {
    return obs ? seg_off<T>() + 12 * sizeof(double)
               : ((size_t)NQS * 6 * QP + (size_t)NSS * 10 * SP + (size_t)NHS * 5 * IP + (size_t)NUS * 3 * SP) *
                         sizeof(T) +
                     (QW + QH) * sizeof(int);
  }
};

__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_all;\n" ::: "memory");
}
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
  if constexpr (sizeof(T) == 4) cp_async4(dst, src); else cp_async8(dst, src);
}

template <typename T, bool SHIFT, int TY, int NS, class V, int FORM, int MODE>
__global__ void __launch_bounds__(512, 1)
    k_step_pipe(const InstDesc<T>* __restrict__ D, const FusedTile* __restrict__ tiles, int ntiles, long long total,
                FusedObs ob) {
  constexpr bool OBS = MODE == kFusedSums;
  using G = PipeGeom<TY, NS>;
  constexpr int QW = G::QW, QP = G::QP, SW = G::SW, SP = G::SP, TX = G::TX;
  constexpr int QSLOT = 6 * QP, SSLOT = 10 * SP, HSLOT = 5 * G::IP, USLOT = 3 * SP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sQ = reinterpret_cast<T*>(smem_raw);
  T* sS = sQ + G::NQS * QSLOT;
  T* sH = sS + G::NSS * SSLOT;
  T* sU = sH + G::NHS * HSLOT;
  int* xmap = reinterpret_cast<int*>(sU + G::NUS * USLOT);
  int* ymap = xmap + QW;
  T* oshare = reinterpret_cast<T*>(smem_raw + G::template obs_off<T>());  // a6 shares [2][IP][12]
  T* oacc = reinterpret_cast<T*>(smem_raw + G::template acc_off<T>());    // sigma-thread sums [NR][2]
  T* xt = reinterpret_cast<T*>(smem_raw + G::template trig_off<T>());     // (cos, sin) of the tile's x
  T* yt = xt + 2 * TX;                                                     // ... and y
  double* oseg = reinterpret_cast<double*>(smem_raw + G::template seg_off<T>());
  const int tid = threadIdx.x;
  auto q6 = [](int p) { return (p + 12) % 6; };
  auto s4 = [](int p) { return (p + 12) % 4; };
  auto h3 = [](int p) { return (p + 12) % 3; };

  const long long begin = (total * blockIdx.x) / gridDim.x;
  const long long end = (total * (blockIdx.x + 1)) / gridDim.x;
  long long it = begin;
  int seg = 0;  // ordinal of the column segment within this block (its a6 slot)
  while (it < end) {
    int lo = 0, hi = ntiles - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tiles[mid].start <= it) lo = mid; else hi = mid - 1;
    }
    const FusedTile tl = tiles[lo];
    const InstDesc<T>& I = D[tl.inst];
    const int nx = I.nx, ny = I.ny, nz = I.nz;
    const long long N = I.N;
    const long long plane = (long long)nx * ny;
    const int zb = (int)(it - tl.start);
    const long long seg_end = end < tl.start + tl.nz ? end : tl.start + tl.nz;
    const int ze = (int)(seg_end - tl.start);
    it = seg_end;
    const Coef<T> cf = I.c;
    const T* __restrict__ qin = I.q_in;
    const T* __restrict__ pin = I.psi_in;
    const T* __restrict__ uin = I.u_in;

    __syncthreads();
    for (int k = tid; k < QW; k += G::NT) xmap[k] = wrapmod(tl.x0 + k - 2, nx);
    for (int k = tid; k < G::QH; k += G::NT) ymap[k] = wrapmod(tl.y0 + k - 2, ny) * nx;
    if constexpr (OBS) {
      for (int k = tid; k < G::NR * 2; k += G::NT) oacc[k] = T(0);
      for (int k = tid; k < 2 * (TX + G::TY); k += G::NT) {  // column k/2 < TX, else row k/2 - TX
        const int e = k >> 1, c = k & 1;
        xt[k] = e < TX ? I.trig[2 * ((tl.x0 + e) % nx) + c] : I.trig[2 * (nx + (tl.y0 + e - TX) % ny) + c];
      }
    }
    __syncthreads();
    // this thread's load sites (at most one Q/psi site and one u site per plane)
    int qoff = 0, uoff = 0;
    if (tid < QP) {
      const int ly = tid / QW, lx = tid - ly * QW;
      qoff = ymap[ly] + xmap[lx];
    }
    if (tid < SP) {
      const int sy = tid / SW, sx = tid - sy * SW;
      uoff = ymap[sy + 1] + xmap[sx + 1];
    }
    auto issue_q = [&](int p) {
      if (tid < QP) {
        T* dst = sQ + q6(p) * QSLOT;
        const long long gs = (long long)wrap_plane(p, nz) * plane + qoff;
#pragma unroll
        for (int f = 0; f < 5; ++f) cp_async_elem(dst + qidx<QP>(f, tid), qin + f * N + gs);
        cp_async_elem(dst + qidx<QP>(5, tid), pin + gs);
      }
    };
    auto issue_u = [&](int p) {
      if (tid < SP) {
        T* dst = sU + s4(p) * USLOT;
        const long long gs = (long long)wrap_plane(p, nz) * plane + uoff;
#pragma unroll
        for (int a = 0; a < 3; ++a) cp_async_elem(dst + uidx<SP>(a, tid), uin + a * N + gs);
      }
    };
    issue_q(zb - 2);
    issue_q(zb - 1);
    issue_q(zb);
    cp_async_commit_wait_all();
    __syncthreads();

    for (int k = zb - 2; k <= ze; ++k) {
      issue_q(k + 3);
      if constexpr (MODE != kFusedLbOnly) issue_u(k + 1);  // the LB half reads no previous u
      if (tid < G::NS) {
        // sigma, mu (and H on interior sites) of plane k+1
#pragma unroll 1
        for (int ss = tid; k + 1 <= ze && ss < SP; ss += G::NS) {
          const int sy = ss / SW, sx = ss - sy * SW;
          SmemFieldsAcc<T, QW, QP> acc;
          acc.qc = (sy + 1) * QW + (sx + 1);
#pragma unroll
          for (int j = 0; j < 3; ++j) acc.pl[j] = sQ + q6(k + j) * QSLOT;
          T q0[5], p0, dq[3][5], lapq[5], dp[3], lapp, hp[6];
          gather_fields<T>(acc, q0, p0, dq, lapq, dp, lapp, hp);
          T H[5], sig[9], mu;
          local_fields<T>(cf, q0, p0, dq, lapq, dp, lapp, hp, H, mu, sig);
          store_sigma<T, SP>(sS + s4(k + 1) * SSLOT, sy * SW + sx, sig, mu);
          if (sx >= 1 && sx <= TX && sy >= 1 && sy <= G::TY) {
            T* hd = sH + h3(k + 1) * HSLOT + (sy - 1) * TX + (sx - 1);
#pragma unroll
            for (int c = 0; c < 5; ++c) hd[c * G::IP] = H[c];
          }
        }
        // a6: the shares of output plane k-2, left by the output warps in the previous phase
        if constexpr (OBS)
          if (k - 2 >= zb) obs_sigma_reduce<T, G>(oshare + ((k - 2) & 1) * G::IP * 12, oacc);
      } else {
        if (k - 1 >= zb) {
          // output of plane z = k-1
          const int z = k - 1;
          const long long zo3[3] = {(long long)wrap_plane(z - 1, nz) * plane, (long long)z * plane,
                                    (long long)wrap_plane(z + 1, nz) * plane};
          // cos, sin of the plane for the a6 centroid sums, read early: its latency hides
          // behind the stencils
          Vec2<T> tz = v2(T(0), T(0));
          if constexpr (OBS) tz = ldg2(I.trig + 2 * (nx + ny + z));
          const int site = tid - G::NS;
          const int tx = site % TX, ty = site / TX;
          T ob6[12] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
          if (site < G::IP && tl.x0 + tx < nx && tl.y0 + ty < ny) {
            SmemUpdateAcc<T, QW, QP, SW, SP> acc;
            acc.qc = (ty + 2) * QW + (tx + 2);
            acc.sc = (ty + 1) * SW + (tx + 1);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
              acc.qpl[j] = sQ + q6(z - 1 + j) * QSLOT;
              acc.spl[j] = sS + s4(z - 1 + j) * SSLOT;
              acc.upl[j] = sU + s4(z - 1 + j) * USLOT;
            }
            T Hs[5];  // read before the stencils: measured faster here than a late read
#pragma unroll
            for (int c = 0; c < 5; ++c) Hs[c] = sH[h3(z) * HSLOT + c * G::IP + site];
            auto hs = [&](T H[5]) {
#pragma unroll
              for (int c = 0; c < 5; ++c) H[c] = Hs[c];
            };
            auto offs = [&](long long zo[3], int pyo[3], int pxo[3]) {
#pragma unroll
              for (int j = 0; j < 3; ++j) {
                zo[j] = zo3[j];
                pyo[j] = ymap[ty + 1 + j];
                pxo[j] = xmap[tx + 1 + j];
              }
            };
            auto trg = [&](Vec2<T>& ctx, Vec2<T>& cty, Vec2<T>& ctz) {
              ctx = lds2(xt + 2 * tx);
              cty = lds2(yt + 2 * ty);
              ctz = tz;
            };
            output_site<T, SHIFT, V, FORM, MODE>(I, cf, acc, offs, hs, trg, GlobalPull<T, V>{I.g_in, N}, ob6);
          }
          if (OBS && site < G::IP) {
            T* dst = oshare + (z & 1) * G::IP * 12 + site * 12;
#pragma unroll
            for (int c = 0; c < 12; c += (sizeof(T) == 4 ? 4 : 2)) {
              if constexpr (sizeof(T) == 4)
                *reinterpret_cast<float4*>(dst + c) = make_float4(ob6[c], ob6[c + 1], ob6[c + 2], ob6[c + 3]);
              else *reinterpret_cast<double2*>(dst + c) = make_double2(ob6[c], ob6[c + 1]);
            }
          }
        }
      }
      cp_async_commit_wait_all();
      __syncthreads();
    }
    if constexpr (OBS) {
      // the last output plane (ze - 1) has not been added up yet
      if (ze - 1 >= zb) obs_sigma_reduce<T, G>(oshare + ((ze - 1) & 1) * G::IP * 12, oacc);
      __syncthreads();
      obs_sigma_values<T, G>(oacc, reinterpret_cast<double*>(smem_raw), oseg);
      __syncthreads();
      obs_segment_write(ob, blockIdx.x * ob.maxseg + seg, oseg);
    }
    ++seg;
  }
  if constexpr (OBS)
    obs_block_end(ob, seg, reinterpret_cast<double*>(smem_raw),
                  [&](int inst) { return SHIFT ? (double)D[inst].c.rho0 * (double)D[inst].N : 0.0; });
}

// ---------------------------------------------------------------- tiled order-parameter half
// The order-parameter half of a sync-coupled or Heun step (after LaunchFused::step_lb), as
// z-marching kernels on the tiles and work split of the fused step (32 x 8 columns, persistent
// blocks): rings of planes with a halo of 1 in shared memory, filled by cp.async one plane
// ahead, one barrier per plane, and the shared per-site functions on them.
//   k_op_tiled<STAGE>: STAGE 0 the update Q + R(Q) (Euler, sync), 1 the Heun predictor
//     (rq = R(Q), qp = Q + rq), 2 the Heun corrector Q + (rq + R(qp))/2, R from gather_op and
//     op_update with u of this step (sync) or of the previous one, H and mu of the scratch;
//   k_fields_pred_tiled: H and mu of the predicted state qp (gather_fields, local_fields) into
//     the sigma scratch, as k_fields<T, true> writes them.
// Ring slots: planes z-1 .. z+2 (the last one arriving).  The values a site reads only at
// itself (H, and in the corrector R(Q) at t and Q, psi at t) arrive the same way, one plane
// ahead, into two slots by plane parity: read from global memory after the stencils, their
// latency stood between the update and the plane barrier.
template <typename T>
struct OpTileGeom {
  static constexpr int TX = 32, TY = 8, NT = TX * TY;
  static constexpr int SW = TX + 2, SH = TY + 2, SP = SW * SH;
  static constexpr int NSLOT = 4;
  static constexpr int QSLOT = 6 * SP, USLOT = 3 * SP, MSLOT = SP;
  __host__ __device__ static constexpr int NSITE(int stage) { return stage == 2 ? 17 : 5; }  // H, rq, Q, psi
  static constexpr size_t site_off = ((size_t)NSLOT * (QSLOT + USLOT + MSLOT) * sizeof(T) + 15) / 16 * 16;
  __host__ __device__ static constexpr size_t maps_off(int stage) {
    return site_off + (size_t)2 * NSITE(stage) * NT * sizeof(T);
  }
  __host__ __device__ static constexpr size_t op_bytes(int stage) { return maps_off(stage) + (SW + SH) * sizeof(int); }
  static constexpr size_t fields_bytes = (size_t)NSLOT * QSLOT * sizeof(T) + (SW + SH) * sizeof(int);
  static constexpr int LD = (SP + NT - 1) / NT;  // plane sites per thread
};

// Neighbour reads of gather_op from the tiles: Q/psi pairs, u, and mu (lane 1 of pair 4).
template <typename T, int SW, int SP>
struct SmemOpAcc {
  const T* qpl[3];
  const T* upl[3];
  const T* mpl[3];
  int sc;
  __device__ __forceinline__ int at(int cx, int cy) const { return sc + cy * SW + cx; }
  __device__ __forceinline__ Vec2<T> pair(int j, int cx, int cy, int cz) const {
    return lds2(qpl[cz + 1] + qidx<SP>(2 * j, at(cx, cy)));
  }
  __device__ __forceinline__ Vec2<T> spair(int, int cx, int cy, int cz) const {
    return Vec2<T>{T(0), mpl[cz + 1][at(cx, cy)]};
  }
  __device__ __forceinline__ Vec2<T> upair(int cx, int cy, int cz) const { return lds2(upl[cz + 1] + 2 * at(cx, cy)); }
  __device__ __forceinline__ T u(int a, int cx, int cy, int cz) const { return upl[cz + 1][uidx<SP>(a, at(cx, cy))]; }
};

// The column segment [zb, ze) of tile tl, plane by plane, for both tiled kernels: load(slot,
// site k, global offset) copies a plane's fields of tile site k; load_site(parity, global offset)
// copies the site-local values of this thread's interior site of a plane (called only for a
// site inside the lattice); work(z, slots of z-1, z, z+1) computes that site.
template <class G, class Load, class LoadSite, class Work>
__device__ __forceinline__ void op_tile_march(const FusedTile& tl, int nx, int ny, int nz, int zb, int ze,
                                              int* xmap, int* ymap, const Load& load, const LoadSite& load_site,
                                              const Work& work) {
  const int tid = threadIdx.x;
  __syncthreads();  // the previous segment is done with the tiles
  for (int k = tid; k < G::SW; k += G::NT) xmap[k] = wrapmod(tl.x0 + k - 1, nx);
  for (int k = tid; k < G::SH; k += G::NT) ymap[k] = wrapmod(tl.y0 + k - 1, ny) * nx;
  __syncthreads();
  int off[G::LD];
#pragma unroll
  for (int r = 0; r < G::LD; ++r) {
    const int k = tid + r * G::NT;
    off[r] = k < G::SP ? ymap[k / G::SW] + xmap[k % G::SW] : 0;
  }
  const long long plane = (long long)nx * ny;
  auto issue = [&](int p) {
    const long long gz = (long long)wrap_plane(p, nz) * plane;
    const int slot = (p + 4 * G::NSLOT) % G::NSLOT;
#pragma unroll
    for (int r = 0; r < G::LD; ++r) {
      const int k = tid + r * G::NT;
      if (k < G::SP) load(slot, k, gz + off[r]);
    }
  };
  const int tx = tid % G::TX, ty = tid / G::TX;
  const bool inside = tl.x0 + tx < nx && tl.y0 + ty < ny;
  const long long soff = (long long)(tl.y0 + ty) * nx + (tl.x0 + tx);
  auto issue_site = [&](int p) {
    if (inside) load_site(p & 1, (long long)p * plane + soff);
  };
  issue(zb - 1);
  issue(zb);
  issue(zb + 1);
  issue_site(zb);
  cp_async_commit_wait_all();
  __syncthreads();
  for (int z = zb; z < ze; ++z) {
    issue(z + 2);
    if (z + 1 < ze) issue_site(z + 1);
    work(z, (z - 1 + 4 * G::NSLOT) % G::NSLOT, z % G::NSLOT, (z + 1) % G::NSLOT);
    cp_async_commit_wait_all();
    __syncthreads();
  }
}

template <typename T, int STAGE>
__global__ void __launch_bounds__(256, (STAGE == 2 || sizeof(T) == 8) ? 2 : 3) k_op_tiled(const InstDesc<T>* __restrict__ D, const FusedTile* __restrict__ tiles,
                                                  int ntiles, long long total, int sync) {
  using G = OpTileGeom<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int NSV = G::NSITE(STAGE);
  T* sQ = reinterpret_cast<T*>(smem_raw);
  T* sU = sQ + G::NSLOT * G::QSLOT;
  T* sM = sU + G::NSLOT * G::USLOT;
  T* sI = reinterpret_cast<T*>(smem_raw + G::site_off);  // site-local values [2][NSV][NT]
  int* xmap = reinterpret_cast<int*>(smem_raw + G::maps_off(STAGE));
  int* ymap = xmap + G::SW;
  const int tid = threadIdx.x, tx = tid % G::TX, ty = tid / G::TX;
  const long long begin = (total * blockIdx.x) / gridDim.x;
  const long long end = (total * (blockIdx.x + 1)) / gridDim.x;
  for (long long it = begin; it < end;) {
    int lo = 0, hi = ntiles - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tiles[mid].start <= it) lo = mid; else hi = mid - 1;
    }
    const FusedTile tl = tiles[lo];
    const InstDesc<T>& I = D[tl.inst];
    const int nx = I.nx, ny = I.ny, nz = I.nz;
    const long long N = I.N;
    const int zb = (int)(it - tl.start);
    const long long seg_end = end < tl.start + tl.nz ? end : tl.start + tl.nz;
    const int ze = (int)(seg_end - tl.start);
    it = seg_end;
    const T* qsrc = STAGE == 2 ? I.qp : I.q_in;
    const T* psrc = STAGE == 2 ? I.qp + 5 * N : I.psi_in;
    const T* usrc = sync ? I.u_out : I.u_in;
    const T* msrc = STAGE == 2 ? I.sig + 5 * N : I.mu;
    const T* hsrc = STAGE == 2 ? I.sig : I.H;
    auto load = [&](int slot, int k, long long gs) {
      T* dq = sQ + slot * G::QSLOT;
#pragma unroll
      for (int f = 0; f < 5; ++f) cp_async_elem(dq + qidx<G::SP>(f, k), qsrc + f * N + gs);
      cp_async_elem(dq + qidx<G::SP>(5, k), psrc + gs);
      T* du = sU + slot * G::USLOT;
#pragma unroll
      for (int a = 0; a < 3; ++a) cp_async_elem(du + uidx<G::SP>(a, k), usrc + a * N + gs);
      cp_async_elem(sM + slot * G::MSLOT + k, msrc + gs);
    };
    auto load_site = [&](int par, long long gs) {
      T* d = sI + par * NSV * G::NT + tid;
#pragma unroll
      for (int k = 0; k < 5; ++k) cp_async_elem(d + k * G::NT, hsrc + k * N + gs);
      if constexpr (STAGE == 2) {
#pragma unroll
        for (int k = 0; k < 6; ++k) cp_async_elem(d + (5 + k) * G::NT, I.rq + k * N + gs);
#pragma unroll
        for (int k = 0; k < 5; ++k) cp_async_elem(d + (11 + k) * G::NT, I.q_in + k * N + gs);
        cp_async_elem(d + 16 * G::NT, I.psi_in + gs);
      }
    };
    auto work = [&](int z, int s0, int s1, int s2) {
      if (tl.x0 + tx >= nx || tl.y0 + ty >= ny) return;
      const T* si = sI + (z & 1) * NSV * G::NT + tid;
      SmemOpAcc<T, G::SW, G::SP> acc;
      const int sl[3] = {s0, s1, s2};
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        acc.qpl[j] = sQ + sl[j] * G::QSLOT;
        acc.upl[j] = sU + sl[j] * G::USLOT;
        acc.mpl[j] = sM + sl[j] * G::MSLOT;
      }
      acc.sc = (ty + 1) * G::SW + (tx + 1);
      T lapmu, Wg[3][3], q0[5], qf[6][5], p0, pf[6], u0[3], uf[6];
      gather_op<T>(acc, lapmu, Wg, q0, qf, p0, pf, u0, uf);
      const long long s = (long long)z * nx * ny + (long long)(tl.y0 + ty) * nx + (tl.x0 + tx);
      T Hs[5];
#pragma unroll
      for (int k = 0; k < 5; ++k) Hs[k] = si[k * G::NT];
      T qn[5], pn;
      if constexpr (STAGE == 0) {
        op_update<T, false>(I.c, lapmu, Wg, q0, qf, p0, pf, u0, uf, Hs, qn, pn);
#pragma unroll
        for (int k = 0; k < 5; ++k) st_out(I.q_out + k * N + s, qn[k]);
        st_out(I.psi_out + s, pn);
      } else if constexpr (STAGE == 1) {
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
        for (int k = 0; k < 5; ++k)
          st_out(I.q_out + k * N + s, si[(11 + k) * G::NT] + T(0.5) * (si[(5 + k) * G::NT] + qn[k]));
        st_out(I.psi_out + s, si[16 * G::NT] + T(0.5) * (si[10 * G::NT] + pn));
      }
    };
    op_tile_march<G>(tl, nx, ny, nz, zb, ze, xmap, ymap, load, load_site, work);
  }
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 2 : 3) k_fields_pred_tiled(const InstDesc<T>* __restrict__ D,
                                                           const FusedTile* __restrict__ tiles, int ntiles,
                                                           long long total) {
  using G = OpTileGeom<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sQ = reinterpret_cast<T*>(smem_raw);
  int* xmap = reinterpret_cast<int*>(sQ + G::NSLOT * G::QSLOT);
  int* ymap = xmap + G::SW;
  const int tid = threadIdx.x, tx = tid % G::TX, ty = tid / G::TX;
  const long long begin = (total * blockIdx.x) / gridDim.x;
  const long long end = (total * (blockIdx.x + 1)) / gridDim.x;
  for (long long it = begin; it < end;) {
    int lo = 0, hi = ntiles - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tiles[mid].start <= it) lo = mid; else hi = mid - 1;
    }
    const FusedTile tl = tiles[lo];
    const InstDesc<T>& I = D[tl.inst];
    const int nx = I.nx, ny = I.ny, nz = I.nz;
    const long long N = I.N;
    const int zb = (int)(it - tl.start);
    const long long seg_end = end < tl.start + tl.nz ? end : tl.start + tl.nz;
    const int ze = (int)(seg_end - tl.start);
    it = seg_end;
    const T* qsrc = I.qp;
    auto load = [&](int slot, int k, long long gs) {
      T* dq = sQ + slot * G::QSLOT;
#pragma unroll
      for (int f = 0; f < 6; ++f) cp_async_elem(dq + qidx<G::SP>(f, k), qsrc + f * N + gs);
    };
    auto work = [&](int z, int s0, int s1, int s2) {
      if (tl.x0 + tx >= nx || tl.y0 + ty >= ny) return;
      SmemFieldsAcc<T, G::SW, G::SP> acc;
      acc.pl[0] = sQ + s0 * G::QSLOT;
      acc.pl[1] = sQ + s1 * G::QSLOT;
      acc.pl[2] = sQ + s2 * G::QSLOT;
      acc.qc = (ty + 1) * G::SW + (tx + 1);
      T q0[5], p0, dq[3][5], lapq[5], dp[3], lapp, hp[6];
      gather_fields<T>(acc, q0, p0, dq, lapq, dp, lapp, hp);
      T H[5], sig[9], mu;
      local_fields<T>(I.c, q0, p0, dq, lapq, dp, lapp, hp, H, mu, sig);
      const long long s = (long long)z * nx * ny + (long long)(tl.y0 + ty) * nx + (tl.x0 + tx);
#pragma unroll
      for (int k = 0; k < 5; ++k) I.sig[k * N + s] = H[k];
      I.sig[5 * N + s] = mu;
    };
    op_tile_march<G>(tl, nx, ny, nz, zb, ze, xmap, ymap, load, [](int, long long) {}, work);
  }
}

// Grid of a tiled order-parameter kernel: every SM times the blocks that fit, at most the units.
// (The FP32 update, predictor and fields kernels are built for three blocks per SM, the
// corrector, with its larger shared-memory slots, for two: 1% faster for Heun than two each.)
template <class K>
int op_tiled_grid(K kernel, size_t smem, long long total) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, 256, smem);
  long long g = (long long)sms * (per > 0 ? per : 1);
  return (int)(g < total ? g : total);
}

template <typename T, bool SHIFT>
cudaError_t LaunchFused<T, SHIFT>::op_tiled(bool heun, bool sync, const InstDesc<T>* d, const FusedTile* t, int nt,
                                            long long total, cudaStream_t s) {
  using G = OpTileGeom<T>;
  // the shared-memory limits are attributes of the functions on the current device (idempotent)
  cudaError_t e =
      cudaFuncSetAttribute(k_op_tiled<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::op_bytes(0));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_op_tiled<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::op_bytes(1));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_op_tiled<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::op_bytes(2));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fields_pred_tiled<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::fields_bytes);
  if (e != cudaSuccess) return e;
  if (!heun) {
    const int g0 = op_tiled_grid(k_op_tiled<T, 0>, G::op_bytes(0), total);
    k_op_tiled<T, 0><<<g0, 256, G::op_bytes(0), s>>>(d, t, nt, total, sync ? 1 : 0);
    return cudaGetLastError();
  }
  const int g1 = op_tiled_grid(k_op_tiled<T, 1>, G::op_bytes(1), total);
  const int gf = op_tiled_grid(k_fields_pred_tiled<T>, G::fields_bytes, total);
  const int g2 = op_tiled_grid(k_op_tiled<T, 2>, G::op_bytes(2), total);
  k_op_tiled<T, 1><<<g1, 256, G::op_bytes(1), s>>>(d, t, nt, total, sync ? 1 : 0);
  k_fields_pred_tiled<T><<<gf, 256, G::fields_bytes, s>>>(d, t, nt, total);
  k_op_tiled<T, 2><<<g2, 256, G::op_bytes(2), s>>>(d, t, nt, total, sync ? 1 : 0);
  return cudaGetLastError();
}

template <typename T, bool SHIFT, int TX, int TY, class V, int FORM>
cudaError_t launch_cfg(const InstDesc<T>* d_desc, const FusedTile* tiles, int ntiles, long long total, int grid,
                       const FusedObs& ob, bool obs, cudaStream_t s) {
  using G = FusedGeom<T, TX, TY>;
  if (obs)
    k_step_fused<T, SHIFT, TX, TY, V, FORM, kFusedSums><<<grid, G::NT, G::bytes(true), s>>>(d_desc, tiles, ntiles,
                                                                                            total, ob);
  else
    k_step_fused<T, SHIFT, TX, TY, V, FORM, kFusedPlain><<<grid, G::NT, G::bytes(false), s>>>(d_desc, tiles, ntiles,
                                                                                              total, ob);
  return cudaGetLastError();
}

// Both kernels of a tile shape (with and without the a6 sums); the launch resources are those
// of the one with the sums (more shared memory), so that both run on the same grid.
template <typename T, bool SHIFT, int TX, int TY, class V, int FORM, bool LB = false>
cudaError_t prepare_cfg(FusedCfg* cfg) {
  using G = FusedGeom<T, TX, TY>;
  auto k0 = k_step_fused<T, SHIFT, TX, TY, V, FORM, kFusedPlain>;
  auto k1 = k_step_fused<T, SHIFT, TX, TY, V, FORM, kFusedSums>;
  auto k2 = k_step_fused<T, SHIFT, TX, TY, V, FORM, kFusedLbOnly>;
  cfg->tx = TX;
  cfg->ty = TY;
  cfg->threads = G::NT;
  cfg->smem = G::bytes(true);
  cudaError_t e = cudaFuncSetAttribute(k0, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::bytes(false));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::bytes(true));
  if (e == cudaSuccess && LB)
    e = cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::bytes(false));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cfg->blocks_per_sm, k1, G::NT, G::bytes(true));
}

// Tile shapes offered to the autotuner: 32x8 (two blocks per SM in FP32), 32x16 and
// 64x8 (one block per SM, fewer redundant halo sites), and the pipelined schedules.  FP64
// only fits 32x8.  The
// D3Q15 and Eq. 9-11 variants come in 32x8 and the pipelined 32x8 schedule with 8 + 8 warps.
template <typename T, bool SHIFT>
int LaunchFused<T, SHIFT>::num_configs() {
  return sizeof(T) == 4 ? 7 : 1;
}

template <typename T, bool SHIFT, int TY, int NS, class V, int FORM, bool LB = false>
cudaError_t prepare_pipe(FusedCfg* cfg) {
  using G = PipeGeom<TY, NS>;
  auto k0 = k_step_pipe<T, SHIFT, TY, NS, V, FORM, kFusedPlain>;
  auto k1 = k_step_pipe<T, SHIFT, TY, NS, V, FORM, kFusedSums>;
  auto k2 = k_step_pipe<T, SHIFT, TY, NS, V, FORM, kFusedLbOnly>;
  cfg->tx = G::TX;
  cfg->ty = G::TY;
  cfg->threads = G::NT;
  cfg->smem = G::template bytes<T>(true);
  cudaError_t e = cudaFuncSetAttribute(k0, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::template bytes<T>(false));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::template bytes<T>(true));
  if (e == cudaSuccess && LB)
    e = cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::template bytes<T>(false));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cfg->blocks_per_sm, k1, G::NT, cfg->smem);
}

template <typename T, bool SHIFT, int TY, int NS, class V, int FORM>
cudaError_t launch_pipe(const InstDesc<T>* d_desc, const FusedTile* tiles, int ntiles, long long total, int grid,
                        const FusedObs& ob, bool obs, cudaStream_t s) {
  using G = PipeGeom<TY, NS>;
  if (obs)
    k_step_pipe<T, SHIFT, TY, NS, V, FORM, kFusedSums><<<grid, G::NT, G::template bytes<T>(true), s>>>(
        d_desc, tiles, ntiles, total, ob);
  else
    k_step_pipe<T, SHIFT, TY, NS, V, FORM, kFusedPlain><<<grid, G::NT, G::template bytes<T>(false), s>>>(
        d_desc, tiles, ntiles, total, ob);
  return cudaGetLastError();
}

// One variant (velocity set V, LB form FORM): cfg_index -> tile shape.
template <typename T, bool SHIFT, class V, int FORM>
struct FusedVariant {
  static constexpr bool ALL = std::is_same<V, VelD3Q19>::value && FORM == 0;
  static cudaError_t prepare(int k, FusedCfg* cfg) {
    if constexpr (sizeof(T) == 4) {
      if constexpr (ALL) {
        if (k == 1) return prepare_cfg<T, SHIFT, 32, 16, V, FORM>(cfg);
        if (k == 2) return prepare_cfg<T, SHIFT, 64, 8, V, FORM>(cfg);
        if (k == 4) return prepare_pipe<T, SHIFT, 8, 192, V, FORM>(cfg);
        if (k == 5) return prepare_pipe<T, SHIFT, 6, 288, V, FORM>(cfg);
        if (k == 6) return prepare_pipe<T, SHIFT, 6, 320, V, FORM>(cfg);
      }
      if (k == 3) return prepare_pipe<T, SHIFT, 8, 256, V, FORM, true>(cfg);
    }
    if (k == 0) return prepare_cfg<T, SHIFT, 32, 8, V, FORM, sizeof(T) == 8>(cfg);
    return k >= 0 && k < LaunchFused<T, SHIFT>::num_configs() ? cudaErrorNotSupported : cudaErrorInvalidValue;
  }
  // the first half of a sync-coupled step: FP32 on the pipelined 32x8 schedule, FP64 on 32x8
  static cudaError_t step_lb(const InstDesc<T>* d, const FusedTile* t, int nt, long long total, int grid,
                             const FusedObs& ob, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
      using G = PipeGeom<8, 256>;
      k_step_pipe<T, SHIFT, 8, 256, V, FORM, kFusedLbOnly><<<grid, G::NT, G::template bytes<T>(false), s>>>(
          d, t, nt, total, ob);
    } else {
      using G = FusedGeom<T, 32, 8>;
      k_step_fused<T, SHIFT, 32, 8, V, FORM, kFusedLbOnly><<<grid, G::NT, G::bytes(false), s>>>(d, t, nt, total, ob);
    }
    return cudaGetLastError();
  }
  static cudaError_t step(int k, const InstDesc<T>* d, const FusedTile* t, int nt, long long total, int grid,
                          const FusedObs& ob, bool obs, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
      if constexpr (ALL) {
        if (k == 1) return launch_cfg<T, SHIFT, 32, 16, V, FORM>(d, t, nt, total, grid, ob, obs, s);
        if (k == 2) return launch_cfg<T, SHIFT, 64, 8, V, FORM>(d, t, nt, total, grid, ob, obs, s);
        if (k == 4) return launch_pipe<T, SHIFT, 8, 192, V, FORM>(d, t, nt, total, grid, ob, obs, s);
        if (k == 5) return launch_pipe<T, SHIFT, 6, 288, V, FORM>(d, t, nt, total, grid, ob, obs, s);
        if (k == 6) return launch_pipe<T, SHIFT, 6, 320, V, FORM>(d, t, nt, total, grid, ob, obs, s);
      }
      if (k == 3) return launch_pipe<T, SHIFT, 8, 256, V, FORM>(d, t, nt, total, grid, ob, obs, s);
    }
    if (k == 0) return launch_cfg<T, SHIFT, 32, 8, V, FORM>(d, t, nt, total, grid, ob, obs, s);
    return cudaErrorInvalidValue;
  }
};

// variant = (velocity set D3Q15 ? 1 : 0) + 2 * (Eq. 9-11 form ? 1 : 0)
template <typename T, bool SHIFT>
cudaError_t LaunchFused<T, SHIFT>::prepare(int variant, int cfg_index, FusedCfg* cfg) {
  switch (variant) {
    case 0: return FusedVariant<T, SHIFT, VelD3Q19, 0>::prepare(cfg_index, cfg);
    case 1: return FusedVariant<T, SHIFT, VelD3Q15, 0>::prepare(cfg_index, cfg);
    case 2: return FusedVariant<T, SHIFT, VelD3Q19, 1>::prepare(cfg_index, cfg);
    case 3: return FusedVariant<T, SHIFT, VelD3Q15, 1>::prepare(cfg_index, cfg);
  }
  return cudaErrorInvalidValue;
}

template <typename T, bool SHIFT>
int LaunchFused<T, SHIFT>::sync_config() {
  return sizeof(T) == 4 ? 3 : 0;
}

template <typename T, bool SHIFT>
cudaError_t LaunchFused<T, SHIFT>::step_lb(int variant, const InstDesc<T>* d_desc, const FusedTile* tiles, int ntiles,
                                           long long total, int grid, const FusedObs& ob, cudaStream_t s) {
  switch (variant) {
    case 0: return FusedVariant<T, SHIFT, VelD3Q19, 0>::step_lb(d_desc, tiles, ntiles, total, grid, ob, s);
    case 1: return FusedVariant<T, SHIFT, VelD3Q15, 0>::step_lb(d_desc, tiles, ntiles, total, grid, ob, s);
    case 2: return FusedVariant<T, SHIFT, VelD3Q19, 1>::step_lb(d_desc, tiles, ntiles, total, grid, ob, s);
    case 3: return FusedVariant<T, SHIFT, VelD3Q15, 1>::step_lb(d_desc, tiles, ntiles, total, grid, ob, s);
  }
  return cudaErrorInvalidValue;
}

template <typename T, bool SHIFT>
cudaError_t LaunchFused<T, SHIFT>::step(int variant, int cfg_index, const InstDesc<T>* d_desc,
                                        const FusedTile* tiles, int ntiles, long long total, int grid,
                                        const FusedObs& ob, bool obs, cudaStream_t s) {
  switch (variant) {
    case 0: return FusedVariant<T, SHIFT, VelD3Q19, 0>::step(cfg_index, d_desc, tiles, ntiles, total, grid, ob, obs, s);
    case 1: return FusedVariant<T, SHIFT, VelD3Q15, 0>::step(cfg_index, d_desc, tiles, ntiles, total, grid, ob, obs, s);
    case 2: return FusedVariant<T, SHIFT, VelD3Q19, 1>::step(cfg_index, d_desc, tiles, ntiles, total, grid, ob, obs, s);
    case 3: return FusedVariant<T, SHIFT, VelD3Q15, 1>::step(cfg_index, d_desc, tiles, ntiles, total, grid, ob, obs, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lbcad
