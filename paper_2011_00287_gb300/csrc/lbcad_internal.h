// lbcad_internal.h -- types shared by the host runtime and the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbcad {

// D3Q19 velocities (rest, six faces, twelve edges), the order published by
// lbcad_lattice().  constexpr so that fully unrolled loops fold them to immediates.
__host__ __device__ constexpr int lat_c(int i, int a) {
  return a == 0 ? (i == 1 ? 1 : i == 2 ? -1 : i == 7 ? 1 : i == 8 ? -1 : i == 9 ? 1 : i == 10 ? -1
                   : i == 11 ? 1 : i == 12 ? -1 : i == 13 ? 1 : i == 14 ? -1 : 0)
       : a == 1 ? (i == 3 ? 1 : i == 4 ? -1 : i == 7 ? 1 : i == 8 ? -1 : i == 9 ? -1 : i == 10 ? 1
                   : i == 15 ? 1 : i == 16 ? -1 : i == 17 ? 1 : i == 18 ? -1 : 0)
                : (i == 5 ? 1 : i == 6 ? -1 : i == 11 ? 1 : i == 12 ? -1 : i == 13 ? -1 : i == 14 ? 1
                   : i == 15 ? 1 : i == 16 ? -1 : i == 17 ? -1 : i == 18 ? 1 : 0);
}
// |c_i|^2: 0 rest, 1 face, 2 edge.
__host__ __device__ constexpr int lat_c2(int i) {
  return lat_c(i, 0) * lat_c(i, 0) + lat_c(i, 1) * lat_c(i, 1) + lat_c(i, 2) * lat_c(i, 2);
}
__host__ __device__ constexpr double lat_w(int i) {
  return lat_c2(i) == 0 ? 1.0 / 3.0 : lat_c2(i) == 1 ? 1.0 / 18.0 : 1.0 / 36.0;
}

// D3Q15 velocities of the LB populations (Sec. 3, Fig. 1): rest, six faces (as in D3Q19),
// eight corners; opposite velocities in adjacent slots.  Weights 2/9, 1/9, 1/72.
__host__ __device__ constexpr int lat15_c(int i, int a) {
  return i == 0 ? 0
       : i <= 6 ? lat_c(i, a)
       : a == 0 ? ((i == 7 || i == 9 || i == 11 || i == 14) ? 1 : -1)
       : a == 1 ? ((i == 7 || i == 9 || i == 12 || i == 13) ? 1 : -1)
                : ((i == 7 || i == 10 || i == 11 || i == 13) ? 1 : -1);
}
__host__ __device__ constexpr double lat15_w(int i) { return i == 0 ? 2.0 / 9.0 : i <= 6 ? 1.0 / 9.0 : 1.0 / 72.0; }

// Velocity sets of the populations as template arguments (the finite-difference stencils
// use D3Q19 in both cases).
struct VelD3Q19 {
  static constexpr int Q = 19;
  __host__ __device__ static constexpr int c(int i, int a) { return lat_c(i, a); }
  __host__ __device__ static constexpr double w(int i) { return lat_w(i); }
};
struct VelD3Q15 {
  static constexpr int Q = 15;
  __host__ __device__ static constexpr int c(int i, int a) { return lat15_c(i, a); }
  __host__ __device__ static constexpr double w(int i) { return lat15_w(i); }
};

// Per-instance coefficients in the compute type.
template <typename T>
struct Coef {
  T tau_inv, guo, rho0;
  T A0, chi0, chis, K, q0, gammaQ, xi, a, b, kphi, M, W, zeta;
};

// One instance of a launch: lattice, state buffers of this step parity, scratch.
template <typename T>
struct InstDesc {
  int nx, ny, nz;
  int vel;         // velocity set of the populations: 0 = D3Q19, 1 = D3Q15
  long long N;
  long long blk0;  // first block of this instance in per-site launches
  long long nblk;  // number of blocks of this instance
  const T* g_in;   // post-collision populations of the previous step [19][N]
  T* g_out;
  const T* q_in;   // [5][N]
  T* q_out;
  const T* psi_in; // [N]
  T* psi_out;
  const T* u_in;   // velocity of the previous step [3][N]
  T* u_out;
  T* sig;          // scratch: stress [9][N]
  T* mu;           // scratch: chemical potential [N]
  T* H;            // scratch: molecular field [5][N]
  T* rq;           // staged path, Heun: right-hand side R(Q, psi) at t [6][N] (Q 5, psi 1)
  T* qp;           // staged path, Heun: predicted Q, psi [6][N]
  const T* trig;   // (cos, sin) of 2 pi x/nx, 2 pi y/ny, 2 pi z/nz: [nx + ny + nz][2] (centroid sums)
  Coef<T> c;
};

// Launchers implemented per precision (lbcad_kernels_f32.cu / _f64.cu).
template <typename T, bool SHIFT>
struct Launch {
  static cudaError_t step(const InstDesc<T>* d_desc, int ninst, long long total_blocks, int bs, cudaStream_t s);
  static cudaError_t fields(const InstDesc<T>* d_desc, int ninst, long long total_blocks, int bs, cudaStream_t s);
  // Staged step: fields -> LB -> order-parameter update (Euler), or fields -> LB ->
  // predictor -> fields at the predicted state -> corrector (Heun).  sync advects with the
  // velocity of this step instead of the previous one.
  // vel: 0 = D3Q19, 1 = D3Q15 populations; form: 0 = whole stress as a body force (Guo),
  // 1 = symmetric stress in the equilibrium, antisymmetric stress as forcing (Eqs. 9-11);
  // stencil: 0 = isotropic D3Q19 finite differences, 1 = fourth-order radius-2 differences.
  static cudaError_t staged(const InstDesc<T>* d_desc, int ninst, long long total_blocks, int bs, bool heun,
                            bool sync, int vel, int form, int stencil, cudaStream_t s);
  static cudaError_t get_fields(const InstDesc<T>& I, uint32_t mask, double* dst, cudaStream_t s);
  static cudaError_t set_fields(const InstDesc<T>& I, uint32_t mask, const double* src, T* g_target,
                                T* q_target, T* psi_target, T* u_target, cudaStream_t s);
  static cudaError_t observables(const InstDesc<T>& I, double* partial, int nblocks, double* out, cudaStream_t s);
};

// One xy tile column of the fused step: instance, tile origin, the instance's nz and the
// first index of this column in the flattened (tile column, z plane) work space.
struct FusedTile {
  int inst, x0, y0, nz;
  long long start;
};

// A tile shape of the fused step and its launch resources.
struct FusedCfg {
  int tx = 0, ty = 0, threads = 0, blocks_per_sm = 0;
  size_t smem = 0;
};

// What a fused step kernel does: the whole step (kFusedPlain), the whole step and the a6 sums
// (kFusedSums), or the LB half of a sync-coupled step (kFusedLbOnly).
constexpr int kFusedPlain = 0, kFusedSums = 1, kFusedLbOnly = 2;

// The FP64 conserved and centroid sums of the fused step (a6).  Each column segment a block
// works on has a slot of 12 partial sums (block b, segment j of the block: slot b * maxseg + j);
// slot_inst[slot] is its instance (-1: unused).  At the end of the kernel each block counts its
// slots on their instances (cnt; the kernel resets it), and the block whose count completes an
// instance sums the instance's slots in a fixed order into latest[inst][12]: mass, sum psi,
// momentum (3), sum phi_c cos (3), sum phi_c sin (3), sum phi_c.
struct FusedObs {
  double* slots;
  const int* slot_inst;
  const int* nslot;    // [ninst] slots of each instance
  const int* slot_lo;  // [ninst] first slot of each instance
  const int* slot_hi;  // [ninst] one past its last slot
  unsigned* cnt;       // [ninst]
  double* latest;      // [ninst][12]
  int maxseg;
};

// The fused one-kernel step (lbcad_fused.cuh), in several tile shapes, for each variant
// of the LB part: variant = (D3Q15 ? 1 : 0) + 2 * (Eq. 9-11 form ? 1 : 0).  prepare returns
// cudaErrorNotSupported for a tile shape the variant does not come in.
template <typename T, bool SHIFT>
struct LaunchFused {
  static int num_configs();
  static cudaError_t prepare(int variant, int cfg_index, FusedCfg* cfg);
  // obs: the kernel that also forms the a6 sums of the new state (FusedObs)
  static cudaError_t step(int variant, int cfg_index, const InstDesc<T>* d_desc, const FusedTile* tiles,
                          int ntiles, long long total, int grid, const FusedObs& ob, bool obs, cudaStream_t s);
  // Sync coupling or Heun: the first half of the step (force, pull, collision, u of this step;
  // H and mu of every site into the scratch), on tile shape sync_config(); op_tiled finishes it.
  static int sync_config();
  static cudaError_t step_lb(int variant, const InstDesc<T>* d_desc, const FusedTile* tiles, int ntiles,
                             long long total, int grid, const FusedObs& ob, cudaStream_t s);
  // The order-parameter half after step_lb as tiled z-marching kernels on the same tiles (32 x 8,
  // the tile shape of sync_config()): the update (Euler), or predictor, fields at the predicted
  // state and corrector (Heun); sync advects with u of this step.
  static cudaError_t op_tiled(bool heun, bool sync, const InstDesc<T>* d_desc, const FusedTile* tiles, int ntiles,
                              long long total, cudaStream_t s);
};

// Buffers of one reverse step of the adjoint (lbcad_adjoint.cuh).
template <typename T>
struct AdjDescHost {
  InstDesc<T> I;                 // state s_t (inputs) and its sigma/mu/H scratch
  const T *lg, *lq, *lp, *lu;    // cotangent of s_{t+1}
  T *A, *Bf, *ls;                // work: 88 + 36 + 15 values per site
  T *og, *oq, *op, *ou;          // cotangent of s_t
  double* pgrad;                 // per-block partial d/dzeta, d/dq0
};

template <typename T, bool SHIFT>
struct LaunchAdj {
  static cudaError_t reverse_step(const AdjDescHost<T>& h, cudaStream_t s);
  static cudaError_t seed(const InstDesc<T>& I, const double dX[3], const double ks[3], const double kc[3], T* lp,
                          cudaStream_t s);
  static int blocks(long long N);
  static cudaError_t export_fields(const InstDesc<T>& I, const T* lam, uint32_t mask, double* dst, cudaStream_t s);
};

// Adds the per-block partial sums of 2 values to total[0..1] (fixed order).
cudaError_t adj_accumulate(const double* pgrad, int nblocks, double* total, cudaStream_t s);

// Sets the message that lbcad_last_error(NULL) returns on this thread.
void set_thread_error(const char* msg);

constexpr int kStepBlock = 256;
constexpr int kObsBlock = 256;
constexpr int kObsMaxBlocks = 1024;
constexpr int kObsRowsPerBlock = 32;  // x rows per block of the separate a6 pass (4 per warp)

}  // namespace lbcad
