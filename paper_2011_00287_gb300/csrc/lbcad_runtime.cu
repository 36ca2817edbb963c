// lbcad_runtime.cu -- host runtime behind the C ABI of include/lbcad.h: parameter
// validation, device memory pool, the seeded initial state, the step loop (optionally
// replayed from a captured CUDA graph), field exchange and FP64 observables.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "lbcad.h"
#include "lbcad_internal.h"
#include "lbcad_validate.h"

using namespace lbcad;

namespace {

thread_local std::string g_create_err;

struct Inst {
  lbcad_grid g;
  lbcad_params p;
  long long N = 0;
  void* gb[2] = {nullptr, nullptr};  // populations, parity 0/1
  void* qb[2] = {nullptr, nullptr};
  void* pb[2] = {nullptr, nullptr};
  void* ub[2] = {nullptr, nullptr};
  void* sig = nullptr;
  void* mu = nullptr;
  void* H = nullptr;
  void* rq = nullptr;  // Heun: right-hand side at t (6 per site)
  void* qp = nullptr;  // Heun: predicted Q, psi (6 per site)
  void* trig = nullptr;  // (cos, sin) of 2 pi x/nx, 2 pi y/ny, 2 pi z/nz for the centroid sums
  long long blk0 = 0, nblk = 0;
};

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (dev >= 0 && dev != prev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

void lbcad::set_thread_error(const char* msg) { g_create_err = msg ? msg : ""; }

struct lbcad_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int prec = LBCAD_FP32;
  lbcad_alloc_fn alloc = nullptr;
  lbcad_free_fn free = nullptr;
  void* user = nullptr;
  std::vector<Inst> inst;
  std::vector<void*> allocs;
  void* desc[2] = {nullptr, nullptr};
  long long total_blocks = 0;
  int64_t step = 0;
  int graph_steps = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  double* obs_partial = nullptr;
  double* obs_out = nullptr;
  double* staging = nullptr;
  size_t staging_bytes = 0;
  int path = LBCAD_PATH_FUSED;
  int integrator = LBCAD_EULER;
  int coupling = LBCAD_LAGGED;
  int vel = LBCAD_D3Q19;          // velocity set of the populations
  int lb_form = LBCAD_LB_BODY_FORCE;
  int stencil = LBCAD_STENCIL_ISO;
  bool scratch_ready = false;
  FusedTile* tiles = nullptr;
  size_t tiles_cap = 0;
  int ntiles = 0;
  long long fused_total = 0;
  int fused_grid = 0;
  int cfg_index = 0;
  FusedCfg cfg;
  // a6 sums of the fused step (see FusedObs): slots per (block, segment), per-instance
  // bookkeeping, and the sums of the latest state; obs_valid while they describe the state
  double* obs_slots = nullptr;
  size_t obs_slots_cap = 0;
  int* obs_map = nullptr;  // slot_inst [nslots], then nslot, slot_lo, slot_hi [ninst each]
  size_t obs_map_cap = 0;
  unsigned* obs_cnt = nullptr;
  double* obs_latest = nullptr;
  int obs_maxseg = 0;
  bool observe = true;     // fused steps form the a6 sums (lbcad_set_observe)
  bool obs_valid = false;
  void* adj_lam = nullptr;  // cotangent of the initial state of the last lbcad_adjoint
  // buffers of lbcad_adjoint, kept for the next call (reused when large enough)
  void* adj_buf[8] = {};
  size_t adj_bytes[8] = {};
  std::string err;
  size_t elem() const { return prec == LBCAD_FP64 ? sizeof(double) : sizeof(float); }
  // the radius-2 stencils run on the staged path only
  bool staged_only() const { return stencil != LBCAD_STENCIL_ISO; }
  // sync coupling or Heun on the fused path: the LB half in the fused kernel on a fixed tile
  // shape, then the order-parameter kernels
  bool sync_split() const { return !staged_only() && (coupling == LBCAD_SYNC || integrator == LBCAD_HEUN); }
  // D3Q19 with the body force: the two-kernel path and the adjoint cover this LB only
  bool default_lb() const { return vel == LBCAD_D3Q19 && lb_form == LBCAD_LB_BODY_FORCE; }
  // variant of the fused kernels (see LaunchFused)
  int fused_variant() const { return (vel == LBCAD_D3Q15 ? 1 : 0) + (lb_form == LBCAD_LB_STRESS_EQ ? 2 : 0); }
  int q() const { return vel == LBCAD_D3Q15 ? 15 : 19; }
};

namespace {

int fail(lbcad_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg; else g_create_err = msg;
  return code;
}

#define CK(ctx, call)                                                                          \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return fail((ctx), LBCAD_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));    \
  } while (0)

void* dev_alloc(lbcad_ctx* c, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  void* p = nullptr;
  if (c->alloc) {
    p = c->alloc(bytes, c->user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) c->allocs.push_back(p);
  return p;
}

// Buffer i of lbcad_adjoint: the one of an earlier call if it is large enough, else a new one
// (the old one stays with the context until it is destroyed).
void* adj_buffer(lbcad_ctx* c, int i, size_t bytes) {
  if (c->adj_buf[i] && c->adj_bytes[i] >= bytes) return c->adj_buf[i];
  void* p = dev_alloc(c, bytes);
  if (p) {
    c->adj_buf[i] = p;
    c->adj_bytes[i] = bytes;
  }
  return p;
}

void release(lbcad_ctx* c) {
  if (!c) return;
  DeviceGuard dg(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  for (void* p : c->allocs) {
    if (c->free) c->free(p, c->user); else cudaFree(p);
  }
  c->allocs.clear();
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

template <typename T>
Coef<T> coefs(const lbcad_params& p) {
  Coef<T> c;
  c.tau_inv = (T)(1.0 / p.tau);
  c.guo = (T)(1.0 - 0.5 / p.tau);
  c.rho0 = (T)p.rho0;
  c.A0 = (T)p.A0; c.chi0 = (T)p.chi0; c.chis = (T)p.chis; c.K = (T)p.K; c.q0 = (T)p.q0;
  c.gammaQ = (T)p.gammaQ; c.xi = (T)p.xi; c.a = (T)p.a; c.b = (T)p.b; c.kphi = (T)p.kphi;
  c.M = (T)p.M; c.W = (T)p.W; c.zeta = (T)p.zeta;
  return c;
}

template <typename T>
InstDesc<T> make_desc(const Inst& I, int parity) {
  InstDesc<T> d;
  std::memset(&d, 0, sizeof(d));
  d.nx = I.g.nx; d.ny = I.g.ny; d.nz = I.g.nz;
  d.vel = (I.p.lattice == LBCAD_D3Q15) ? 1 : 0;
  d.N = I.N;
  d.blk0 = I.blk0;
  d.nblk = I.nblk;
  const int a = parity, b = parity ^ 1;
  d.g_in = (const T*)I.gb[a]; d.g_out = (T*)I.gb[b];
  d.q_in = (const T*)I.qb[a]; d.q_out = (T*)I.qb[b];
  d.psi_in = (const T*)I.pb[a]; d.psi_out = (T*)I.pb[b];
  d.u_in = (const T*)I.ub[a]; d.u_out = (T*)I.ub[b];
  d.sig = (T*)I.sig; d.mu = (T*)I.mu; d.H = (T*)I.H;
  d.rq = (T*)I.rq; d.qp = (T*)I.qp;
  d.trig = (const T*)I.trig;
  d.c = coefs<T>(I.p);
  return d;
}

// SplitMix64 (Steele, Lea & Flood 2014): output number k of the stream started at seed.
inline uint64_t splitmix64(uint64_t seed, uint64_t k) {
  uint64_t z = seed + k * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

inline double unit_noise(uint64_t seed, int inst, long long site, int comp) {
  const uint64_t k = 1ULL + ((uint64_t)inst << 40) + 5ULL * (uint64_t)site + (uint64_t)comp;
  return 2.0 * ((double)(splitmix64(seed, k) >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
}

// Seeded initial droplet in FP64 on the host: psi = tanh((R - r)/2); a cholesteric
// helix about z of order S0 plus noise inside r < R; Q = 0 outside.
void init_host(const lbcad_grid& g, const lbcad_params& p, uint64_t seed, int inst, std::vector<double>& q5,
               std::vector<double>& psi) {
  const long long N = (long long)g.nx * g.ny * g.nz;
  q5.assign(5 * N, 0.0);
  psi.assign(N, 0.0);
  for (int z = 0; z < g.nz; ++z)
    for (int y = 0; y < g.ny; ++y)
      for (int x = 0; x < g.nx; ++x) {
        const long long s = x + (long long)g.nx * (y + (long long)g.ny * z);
        const double dx = x - p.centre[0], dy = y - p.centre[1], dz = z - p.centre[2];
        const double r = std::sqrt(dx * dx + dy * dy + dz * dz);
        psi[s] = std::tanh((p.R - r) / 2.0);
        if (r < p.R) {
          const double n0 = std::cos(p.q0 * dz), n1 = std::sin(p.q0 * dz);
          double Q[5] = {p.S0 * (n0 * n0 - 1.0 / 3.0), p.S0 * (n0 * n1), 0.0, p.S0 * (n1 * n1 - 1.0 / 3.0), 0.0};
          for (int k = 0; k < 5; ++k) q5[k * N + s] = Q[k] + p.noise * unit_noise(seed, inst, s, k);
        }
      }
}

// v into p[0 .. n) (the rest populations of the initial state, on the device).
template <typename T>
__global__ void k_fill(T* __restrict__ p, long long n, T v) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
    p[k] = v;
}

template <typename T>
int upload_init(lbcad_ctx* c, Inst& I, uint64_t seed, int idx) {
  std::vector<double> q5, psi;
  init_host(I.g, I.p, seed, idx, q5, psi);
  const long long N = I.N;
  std::vector<T> tq(5 * N), tp(N);
  for (long long k = 0; k < 5 * N; ++k) tq[k] = (T)q5[k];
  for (long long k = 0; k < N; ++k) tp[k] = (T)psi[k];
  // populations at rest: w_i rho0, which the shifted FP32 storage holds as 0
  const bool shifted = (c->prec == LBCAD_FP32);
  const int q = c->q();
  T* g0 = (T*)I.gb[0];
  if (shifted) {
    CK(c, cudaMemsetAsync(g0, 0, q * N * sizeof(T), c->stream));
  } else {
    for (int i = 0; i < q; ++i) {
      const double w = (q == 15) ? lat15_w(i) : lat_w(i);
      k_fill<T><<<1024, 256, 0, c->stream>>>(g0 + i * N, N, (T)(w * I.p.rho0));
      CK(c, cudaGetLastError());
    }
  }
  CK(c, cudaMemcpyAsync(I.qb[0], tq.data(), 5 * N * sizeof(T), cudaMemcpyHostToDevice, c->stream));
  CK(c, cudaMemcpyAsync(I.pb[0], tp.data(), N * sizeof(T), cudaMemcpyHostToDevice, c->stream));
  CK(c, cudaMemsetAsync(I.ub[0], 0, 3 * N * sizeof(T), c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return LBCAD_OK;
}

int upload_descs(lbcad_ctx* c);
int prepare_fused(lbcad_ctx* c, int cfg_index);
int ensure_scratch(lbcad_ctx* c);
cudaError_t launch_fused_lb(lbcad_ctx* c, int par);

int create_impl(int n, const lbcad_grid* grids, const lbcad_params* params, uint64_t seed, lbcad_ctx** out) {
  g_create_err.clear();
  if (!out) return fail(nullptr, LBCAD_E_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n < 1 || !grids || !params) return fail(nullptr, LBCAD_E_INVALID_ARG, "need n >= 1 grids and params");
  for (int i = 0; i < n; ++i) {
    std::string v = validate(grids[i], params[i]);
    if (!v.empty()) return fail(nullptr, LBCAD_E_INVALID_ARG, "instance " + std::to_string(i) + ": " + v);
    if (params[i].precision != params[0].precision)
      return fail(nullptr, LBCAD_E_INVALID_ARG, "all instances must share one precision");
    if (params[i].integrator != params[0].integrator || params[i].coupling != params[0].coupling)
      return fail(nullptr, LBCAD_E_INVALID_ARG, "all instances must share one integrator and one coupling");
    if (params[i].lattice != params[0].lattice || params[i].lb_form != params[0].lb_form ||
        params[i].stencil != params[0].stencil)
      return fail(nullptr, LBCAD_E_INVALID_ARG, "all instances must share one lattice, lb_form and stencil");
  }
  lbcad_ctx* c = new (std::nothrow) lbcad_ctx();
  if (!c) return fail(nullptr, LBCAD_E_OOM, "host allocation failed");
  const lbcad_params& p0 = params[0];
  c->prec = p0.precision;
  c->integrator = p0.integrator;
  c->coupling = p0.coupling;
  c->vel = p0.lattice;
  c->lb_form = p0.lb_form;
  c->stencil = p0.stencil;
  c->alloc = p0.alloc;
  c->free = p0.free;
  c->user = p0.alloc_user;
  if ((c->alloc == nullptr) != (c->free == nullptr)) {
    delete c;
    return fail(nullptr, LBCAD_E_INVALID_ARG, "alloc and free callbacks must be given together");
  }
  if (p0.device >= 0) {
    c->device = p0.device;
  } else if (cudaGetDevice(&c->device) != cudaSuccess) {
    delete c;
    return fail(nullptr, LBCAD_E_CUDA, "no CUDA device");
  }
  DeviceGuard dg(c->device);
  int code = LBCAD_OK;
  auto bail = [&](int cd, const std::string& m) {
    g_create_err = m.empty() ? c->err : m;
    release(c);
    delete c;
    return cd;
  };
  if (p0.stream) {
    c->stream = (cudaStream_t)p0.stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess)
      return bail(LBCAD_E_CUDA, "cudaStreamCreateWithFlags failed");
    c->own_stream = true;
  }
  const size_t es = c->elem();
  long long blk = 0;
  long long maxN = 0;
  c->inst.resize(n);
  for (int i = 0; i < n; ++i) {
    Inst& I = c->inst[i];
    I.g = grids[i];
    I.p = params[i];
    I.N = (long long)I.g.nx * I.g.ny * I.g.nz;
    maxN = I.N > maxN ? I.N : maxN;
    I.blk0 = blk;
    I.nblk = (I.N + kStepBlock - 1) / kStepBlock;
    blk += I.nblk;
    for (int par = 0; par < 2; ++par) {
      I.gb[par] = dev_alloc(c, (size_t)c->q() * I.N * es);
      I.qb[par] = dev_alloc(c, 5 * I.N * es);
      I.pb[par] = dev_alloc(c, I.N * es);
      I.ub[par] = dev_alloc(c, 3 * I.N * es);
      if (!I.gb[par] || !I.qb[par] || !I.pb[par] || !I.ub[par]) return bail(LBCAD_E_OOM, "device allocation failed");
    }
    const int L = I.g.nx + I.g.ny + I.g.nz;
    I.trig = dev_alloc(c, 2 * (size_t)L * es);
    if (!I.trig) return bail(LBCAD_E_OOM, "device allocation failed");
    std::vector<double> tr(2 * (size_t)L);
    const int len[3] = {I.g.nx, I.g.ny, I.g.nz};
    for (int a = 0, k = 0; a < 3; ++a)
      for (int x = 0; x < len[a]; ++x, ++k) {
        const double ph = 2.0 * M_PI * (double)x / (double)len[a];
        tr[2 * k] = std::cos(ph);
        tr[2 * k + 1] = std::sin(ph);
      }
    cudaError_t te;
    std::vector<float> tf(tr.begin(), tr.end());
    if (c->prec == LBCAD_FP64)
      te = cudaMemcpyAsync(I.trig, tr.data(), tr.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    else
      te = cudaMemcpyAsync(I.trig, tf.data(), tf.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream);
    if (te == cudaSuccess) te = cudaStreamSynchronize(c->stream);
    if (te != cudaSuccess) return bail(LBCAD_E_CUDA, std::string("trig table upload: ") + cudaGetErrorString(te));
  }
  c->obs_cnt = (unsigned*)dev_alloc(c, n * sizeof(unsigned));
  c->obs_latest = (double*)dev_alloc(c, (size_t)n * 12 * sizeof(double));
  if (!c->obs_cnt || !c->obs_latest) return bail(LBCAD_E_OOM, "device allocation failed");
  if (cudaMemsetAsync(c->obs_cnt, 0, n * sizeof(unsigned), c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return bail(LBCAD_E_CUDA, "a6 counter initialisation failed");
  c->total_blocks = blk;
  if (blk >= (1LL << 31)) return bail(LBCAD_E_INVALID_ARG, "too many blocks for one launch");
  const size_t dsz = (c->prec == LBCAD_FP64 ? sizeof(InstDesc<double>) : sizeof(InstDesc<float>)) * n;
  for (int par = 0; par < 2; ++par) {
    c->desc[par] = dev_alloc(c, dsz);
    if (!c->desc[par]) return bail(LBCAD_E_OOM, "device allocation failed");
  }
  c->obs_partial = (double*)dev_alloc(c, kObsMaxBlocks * 12 * sizeof(double));
  c->obs_out = (double*)dev_alloc(c, 12 * sizeof(double));
  if (!c->obs_partial || !c->obs_out) return bail(LBCAD_E_OOM, "device allocation failed");
  if (upload_descs(c) != LBCAD_OK) return bail(LBCAD_E_CUDA, "");
  // default tile shape: the pipelined 32x8 schedule in FP32 (the fastest candidate from 16^3 to
  // 128^3; the one sync coupling and Heun run on), 32x8 in FP64 (the only one)
  const int cfg0 = c->prec == LBCAD_FP64 ? LaunchFused<double, false>::sync_config()
                                         : LaunchFused<float, true>::sync_config();
  if ((code = prepare_fused(c, cfg0)) != LBCAD_OK) return bail(code, "");
  if (c->staged_only() || c->sync_split()) {
    if ((code = ensure_scratch(c)) != LBCAD_OK) return bail(code, "");
  }
  if (c->staged_only()) c->path = LBCAD_PATH_STAGED;
  for (int i = 0; i < n; ++i) {
    code = (c->prec == LBCAD_FP64) ? upload_init<double>(c, c->inst[i], seed, i)
                                   : upload_init<float>(c, c->inst[i], seed, i);
    if (code != LBCAD_OK) return bail(code, "");
  }
  *out = c;
  return LBCAD_OK;
}

int upload_descs(lbcad_ctx* c) {
  const int n = (int)c->inst.size();
  for (int par = 0; par < 2; ++par) {
    if (c->prec == LBCAD_FP64) {
      std::vector<InstDesc<double>> h(n);
      for (int i = 0; i < n; ++i) h[i] = make_desc<double>(c->inst[i], par);
      CK(c, cudaMemcpyAsync(c->desc[par], h.data(), n * sizeof(h[0]), cudaMemcpyHostToDevice, c->stream));
      CK(c, cudaStreamSynchronize(c->stream));
    } else {
      std::vector<InstDesc<float>> h(n);
      for (int i = 0; i < n; ++i) h[i] = make_desc<float>(c->inst[i], par);
      CK(c, cudaMemcpyAsync(c->desc[par], h.data(), n * sizeof(h[0]), cudaMemcpyHostToDevice, c->stream));
      CK(c, cudaStreamSynchronize(c->stream));
    }
  }
  return LBCAD_OK;
}

// Scratch (sigma, mu, H per site) of the two-kernel and staged paths, allocated on first
// use; Heun contexts also hold the right-hand side at t and the predicted state.
int ensure_scratch(lbcad_ctx* c) {
  if (c->scratch_ready) return LBCAD_OK;
  const size_t es = c->elem();
  for (Inst& I : c->inst) {
    I.sig = dev_alloc(c, 9 * I.N * es);
    I.mu = dev_alloc(c, I.N * es);
    I.H = dev_alloc(c, 5 * I.N * es);
    if (!I.sig || !I.mu || !I.H) return fail(c, LBCAD_E_OOM, "scratch allocation failed");
    if (c->integrator == LBCAD_HEUN) {
      I.rq = dev_alloc(c, 6 * I.N * es);
      I.qp = dev_alloc(c, 6 * I.N * es);
      if (!I.rq || !I.qp) return fail(c, LBCAD_E_OOM, "scratch allocation failed");
    }
  }
  c->scratch_ready = true;
  return upload_descs(c);
}

// Tile columns of the fused step for tile shape `cfg_index` and its persistent grid size.
int prepare_fused(lbcad_ctx* c, int cfg_index) {
  FusedCfg cfg;
  const int v = c->fused_variant();
  cudaError_t e = (c->prec == LBCAD_FP64) ? LaunchFused<double, false>::prepare(v, cfg_index, &cfg)
                                          : LaunchFused<float, true>::prepare(v, cfg_index, &cfg);
  if (e == cudaErrorNotSupported)
    return fail(c, LBCAD_E_UNSUPPORTED, "this velocity set and LB form do not come in that tile shape");
  if (e != cudaSuccess) return fail(c, LBCAD_E_CUDA, std::string("fused kernel set-up: ") + cudaGetErrorString(e));
  if (cfg.blocks_per_sm < 1) return fail(c, LBCAD_E_UNSUPPORTED, "fused tile shape does not fit on an SM");
  std::vector<FusedTile> t;
  long long start = 0;
  for (int i = 0; i < (int)c->inst.size(); ++i) {
    const Inst& I = c->inst[i];
    for (int y0 = 0; y0 < I.g.ny; y0 += cfg.ty)
      for (int x0 = 0; x0 < I.g.nx; x0 += cfg.tx) {
        t.push_back(FusedTile{i, x0, y0, I.g.nz, start});
        start += I.g.nz;
      }
  }
  if (t.size() > c->tiles_cap) {
    c->tiles = (FusedTile*)dev_alloc(c, t.size() * sizeof(FusedTile));
    if (!c->tiles) return fail(c, LBCAD_E_OOM, "tile list allocation failed");
    c->tiles_cap = t.size();
  }
  CK(c, cudaMemcpyAsync(c->tiles, t.data(), t.size() * sizeof(FusedTile), cudaMemcpyHostToDevice, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  int sms = 0;
  CK(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
  long long grid = (long long)sms * cfg.blocks_per_sm;
  if (grid > start) grid = start;
  // the column segments of each block, split exactly as the kernels split them: slot
  // (block, segment) -> instance, and each instance's slot count and range
  const int ninst = (int)c->inst.size();
  std::vector<std::vector<int>> seg_inst(grid);
  int maxseg = 1;
  for (long long b = 0; b < grid; ++b) {
    const long long begin = (start * b) / grid, end = (start * (b + 1)) / grid;
    for (long long it = begin; it < end;) {
      int lo = 0, hi = (int)t.size() - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (t[mid].start <= it) lo = mid; else hi = mid - 1;
      }
      const long long seg_end = std::min(end, t[lo].start + t[lo].nz);
      seg_inst[b].push_back(t[lo].inst);
      it = seg_end;
    }
    maxseg = std::max(maxseg, (int)seg_inst[b].size());
  }
  const size_t nslots = (size_t)grid * maxseg;
  std::vector<int> map(nslots + 3 * (size_t)ninst, -1);
  int* nslot = map.data() + nslots;
  int* slot_lo = nslot + ninst;
  int* slot_hi = slot_lo + ninst;
  for (int i = 0; i < ninst; ++i) nslot[i] = 0;
  for (long long b = 0; b < grid; ++b)
    for (size_t j = 0; j < seg_inst[b].size(); ++j) {
      const int sl = (int)(b * maxseg + j), i = seg_inst[b][j];
      map[sl] = i;
      if (nslot[i]++ == 0) slot_lo[i] = sl;
      slot_hi[i] = sl + 1;
    }
  for (int i = 0; i < ninst; ++i)
    if (nslot[i] == 0) return fail(c, LBCAD_E_INVALID_ARG, "an instance has no fused work");
  if (nslots * 12 > c->obs_slots_cap) {
    c->obs_slots = (double*)dev_alloc(c, nslots * 12 * sizeof(double));
    if (!c->obs_slots) return fail(c, LBCAD_E_OOM, "a6 slot allocation failed");
    c->obs_slots_cap = nslots * 12;
  }
  if (map.size() > c->obs_map_cap) {
    c->obs_map = (int*)dev_alloc(c, map.size() * sizeof(int));
    if (!c->obs_map) return fail(c, LBCAD_E_OOM, "a6 slot map allocation failed");
    c->obs_map_cap = map.size();
  }
  CK(c, cudaMemcpyAsync(c->obs_map, map.data(), map.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  // the kernels leave the per-instance counters at zero; reset them here as well, so that a
  // launch that failed part-way cannot shift the next sums
  CK(c, cudaMemsetAsync(c->obs_cnt, 0, (size_t)ninst * sizeof(unsigned), c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  c->obs_maxseg = maxseg;
  c->obs_valid = false;
  c->ntiles = (int)t.size();
  c->fused_total = start;
  c->fused_grid = (int)grid;
  c->cfg_index = cfg_index;
  c->cfg = cfg;
  return LBCAD_OK;
}

cudaError_t launch_fused(lbcad_ctx* c, int par) {
  const int v = c->fused_variant();
  const int ninst = (int)c->inst.size();
  const size_t nslots = (size_t)c->fused_grid * c->obs_maxseg;
  FusedObs ob;
  ob.slots = c->obs_slots;
  ob.slot_inst = c->obs_map;
  ob.nslot = c->obs_map + nslots;
  ob.slot_lo = ob.nslot + ninst;
  ob.slot_hi = ob.slot_lo + ninst;
  ob.cnt = c->obs_cnt;
  ob.latest = c->obs_latest;
  ob.maxseg = c->obs_maxseg;
  if (c->prec == LBCAD_FP64)
    return LaunchFused<double, false>::step(v, c->cfg_index, (const InstDesc<double>*)c->desc[par], c->tiles,
                                            c->ntiles, c->fused_total, c->fused_grid, ob, c->observe, c->stream);
  return LaunchFused<float, true>::step(v, c->cfg_index, (const InstDesc<float>*)c->desc[par], c->tiles, c->ntiles,
                                        c->fused_total, c->fused_grid, ob, c->observe, c->stream);
}

cudaError_t launch_fused_lb(lbcad_ctx* c, int par) {
  const int v = c->fused_variant();
  FusedObs ob{};  // the LB half forms no sums
  if (c->prec == LBCAD_FP64)
    return LaunchFused<double, false>::step_lb(v, (const InstDesc<double>*)c->desc[par], c->tiles, c->ntiles,
                                               c->fused_total, c->fused_grid, ob, c->stream);
  return LaunchFused<float, true>::step_lb(v, (const InstDesc<float>*)c->desc[par], c->tiles, c->ntiles,
                                           c->fused_total, c->fused_grid, ob, c->stream);
}

void drop_graph(lbcad_ctx* c) {
  if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
  if (c->graph) { cudaGraphDestroy(c->graph); c->graph = nullptr; }
}

int launch_steps(lbcad_ctx* c, int64_t n) {
  for (int64_t k = 0; k < n; ++k) {
    const int par = (int)(c->step & 1);
    cudaError_t e;
    const bool heun = c->integrator == LBCAD_HEUN, sync = c->coupling == LBCAD_SYNC;
    if (c->path == LBCAD_PATH_FUSED && c->sync_split()) {
      // the LB half in the fused kernel, then the order-parameter half as tiled kernels on the
      // same tiles (Euler: the update; Heun: predictor, fields at the predicted state, corrector)
      e = launch_fused_lb(c, par);
      if (e == cudaSuccess)
        e = (c->prec == LBCAD_FP64)
                ? LaunchFused<double, false>::op_tiled(heun, sync, (const InstDesc<double>*)c->desc[par], c->tiles,
                                                       c->ntiles, c->fused_total, c->stream)
                : LaunchFused<float, true>::op_tiled(heun, sync, (const InstDesc<float>*)c->desc[par], c->tiles,
                                                     c->ntiles, c->fused_total, c->stream);
    } else if (c->path == LBCAD_PATH_FUSED) {
      e = launch_fused(c, par);
    } else if (c->path == LBCAD_PATH_STAGED) {
      e = (c->prec == LBCAD_FP64)
              ? Launch<double, false>::staged((const InstDesc<double>*)c->desc[par], (int)c->inst.size(),
                                              c->total_blocks, kStepBlock, heun, sync, c->vel, c->lb_form,
                                              c->stencil, c->stream)
              : Launch<float, true>::staged((const InstDesc<float>*)c->desc[par], (int)c->inst.size(),
                                            c->total_blocks, kStepBlock, heun, sync, c->vel, c->lb_form,
                                            c->stencil, c->stream);
    } else if (c->prec == LBCAD_FP64)
      e = Launch<double, false>::step((const InstDesc<double>*)c->desc[par], (int)c->inst.size(), c->total_blocks,
                                      kStepBlock, c->stream);
    else
      e = Launch<float, true>::step((const InstDesc<float>*)c->desc[par], (int)c->inst.size(), c->total_blocks,
                                    kStepBlock, c->stream);
    if (e != cudaSuccess) return fail(c, LBCAD_E_CUDA, std::string("step launch: ") + cudaGetErrorString(e));
    c->step++;
  }
  return LBCAD_OK;
}

template <typename T>
InstDesc<T> desc_now(const lbcad_ctx* c, int inst) {
  return make_desc<T>(c->inst[inst], (int)(c->step & 1));
}

int ensure_staging(lbcad_ctx* c, size_t bytes) {
  if (c->staging_bytes >= bytes) return LBCAD_OK;
  // the old buffer stays in the pool until destroy; staging only grows
  void* p = dev_alloc(c, bytes);
  if (!p) return fail(c, LBCAD_E_OOM, "staging allocation failed");
  c->staging = (double*)p;
  c->staging_bytes = bytes;
  return LBCAD_OK;
}

int ncomp_of(uint32_t mask, int q = 19) {
  return ((mask & LBCAD_FIELD_G) ? q : 0) + ((mask & LBCAD_FIELD_RHO) ? 1 : 0) + ((mask & LBCAD_FIELD_U) ? 3 : 0) +
         ((mask & LBCAD_FIELD_Q) ? 5 : 0) + ((mask & LBCAD_FIELD_PSI) ? 1 : 0);
}

}  // namespace

extern "C" {

int lbcad_lattice(int32_t* c57, double* w19) {
  if (!c57 || !w19) return LBCAD_E_INVALID_ARG;
  for (int i = 0; i < 19; ++i) {
    for (int a = 0; a < 3; ++a) c57[3 * i + a] = lat_c(i, a);
    w19[i] = lat_w(i);
  }
  return LBCAD_OK;
}

int lbcad_velocity_set(int32_t lattice, int32_t* c, double* w) {
  if (!c || !w || (lattice != LBCAD_D3Q19 && lattice != LBCAD_D3Q15)) return LBCAD_E_INVALID_ARG;
  const int q = (lattice == LBCAD_D3Q15) ? 15 : 19;
  for (int i = 0; i < q; ++i) {
    for (int a = 0; a < 3; ++a) c[3 * i + a] = (q == 15) ? lat15_c(i, a) : lat_c(i, a);
    w[i] = (q == 15) ? lat15_w(i) : lat_w(i);
  }
  return q;
}

int lbcad_create(const lbcad_grid* grid, const lbcad_params* params, uint64_t seed, lbcad_ctx** out) {
  return create_impl(1, grid, params, seed, out);
}

int lbcad_create_batch(int32_t n, const lbcad_grid* grids, const lbcad_params* params, uint64_t seed,
                       lbcad_ctx** out) {
  return create_impl(n, grids, params, seed, out);
}

int lbcad_set_path(lbcad_ctx* c, int32_t path) {
  if (!c) return LBCAD_E_INVALID_ARG;
  if (path != LBCAD_PATH_FUSED && path != LBCAD_PATH_TWO_KERNEL && path != LBCAD_PATH_STAGED)
    return fail(c, LBCAD_E_INVALID_ARG, "unknown path");
  if (path != LBCAD_PATH_STAGED && c->staged_only())
    return fail(c, LBCAD_E_UNSUPPORTED, "radius-2 contexts run on the staged path only");
  if (path == LBCAD_PATH_TWO_KERNEL && (!c->default_lb() || c->sync_split()))
    return fail(c, LBCAD_E_UNSUPPORTED, "the two-kernel path covers the Euler, lagged step of D3Q19 with the body force");
  DeviceGuard dg(c->device);
  if (path != LBCAD_PATH_FUSED) {
    int r = ensure_scratch(c);
    if (r) return r;
  }
  if (path != c->path) {
    if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
    if (c->graph) { cudaGraphDestroy(c->graph); c->graph = nullptr; }
    c->path = path;
    c->obs_valid = false;
  }
  return LBCAD_OK;
}

int lbcad_autotune(lbcad_ctx* c, int32_t reps, int32_t* chosen, float* ms_per_cfg, int32_t ncfg) {
  if (!c || reps < 1) return LBCAD_E_INVALID_ARG;
  if (c->staged_only()) return fail(c, LBCAD_E_UNSUPPORTED, "tile shapes belong to the fused path (Euler, lagged)");
  if (c->sync_split()) return fail(c, LBCAD_E_UNSUPPORTED, "sync coupling and Heun run on one fixed fused tile shape");
  DeviceGuard dg(c->device);
  const int n = (c->prec == LBCAD_FP64) ? LaunchFused<double, false>::num_configs()
                                        : LaunchFused<float, true>::num_configs();
  const int par = (int)(c->step & 1);
  cudaEvent_t e0, e1;
  CK(c, cudaEventCreate(&e0));
  CK(c, cudaEventCreate(&e1));
  // three rounds over the candidates, each candidate timed over `reps` launches after one
  // untimed launch; a candidate's time is its best round (rounds interleave the candidates,
  // so a drift of the clocks during tuning does not favour one of them)
  constexpr int kRounds = 3;
  std::vector<float> best_of(n, -1.f);
  for (int round = 0; round < kRounds; ++round) {
    for (int k = 0; k < n; ++k) {
      if (round > 0 && best_of[k] < 0.f) continue;  // does not fit
      if (prepare_fused(c, k) != LBCAD_OK) continue;
      float ms = -1.f;
      cudaError_t e = launch_fused(c, par);
      if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
      for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_fused(c, par);
      if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) ms /= reps;
      if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return fail(c, LBCAD_E_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
      }
      if (best_of[k] < 0.f || ms < best_of[k]) best_of[k] = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int best = -1;
  for (int k = 0; k < n; ++k) {
    if (best_of[k] >= 0.f && (best < 0 || best_of[k] < best_of[best])) best = k;
    if (ms_per_cfg && k < ncfg) ms_per_cfg[k] = best_of[k];
  }
  if (best < 0) return fail(c, LBCAD_E_UNSUPPORTED, "no fused tile shape fits");
  int r = prepare_fused(c, best);
  if (r) return r;
  drop_graph(c);
  if (chosen) *chosen = best;
  return LBCAD_OK;
}

int lbcad_set_tiles(lbcad_ctx* c, int32_t cfg) {
  if (!c) return LBCAD_E_INVALID_ARG;
  if (c->staged_only()) return fail(c, LBCAD_E_UNSUPPORTED, "tile shapes belong to the fused path (Euler, lagged)");
  if (c->sync_split()) return fail(c, LBCAD_E_UNSUPPORTED, "sync coupling and Heun run on one fixed fused tile shape");
  DeviceGuard dg(c->device);
  const int n = (c->prec == LBCAD_FP64) ? LaunchFused<double, false>::num_configs()
                                        : LaunchFused<float, true>::num_configs();
  if (cfg < 0 || cfg >= n) return fail(c, LBCAD_E_INVALID_ARG, "tile shape index out of range");
  int r = prepare_fused(c, cfg);
  if (r) return r;
  drop_graph(c);
  return LBCAD_OK;
}

int lbcad_set_observe(lbcad_ctx* c, int32_t on) {
  if (!c || (on != 0 && on != 1)) return LBCAD_E_INVALID_ARG;
  if (c->observe != (on == 1)) {
    c->observe = on == 1;
    drop_graph(c);
    c->obs_valid = false;
  }
  return LBCAD_OK;
}

int lbcad_set_graph(lbcad_ctx* c, int32_t steps_per_graph) {
  if (!c) return LBCAD_E_INVALID_ARG;
  // a replay must leave the ping-pong parity unchanged, so a graph holds an even number of steps
  if (steps_per_graph < 0 || (steps_per_graph & 1))
    return fail(c, LBCAD_E_INVALID_ARG, "steps_per_graph must be 0 or a positive even number");
  DeviceGuard dg(c->device);
  if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
  if (c->graph) { cudaGraphDestroy(c->graph); c->graph = nullptr; }
  c->graph_steps = steps_per_graph;
  return LBCAD_OK;
}

int lbcad_step(lbcad_ctx* c, int64_t n) {
  if (!c || n < 0) return LBCAD_E_INVALID_ARG;
  DeviceGuard dg(c->device);
  int64_t left = n;
  if (c->graph_steps > 0) {
    if ((c->step & 1) && left > 0) {
      int r = launch_steps(c, 1);
      if (r) return r;
      left--;
    }
    while (left >= c->graph_steps) {
      if (!c->gexec) {
        const int64_t step0 = c->step;
        CK(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        int r = launch_steps(c, c->graph_steps);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        c->step = step0;
        if (r) { if (g) cudaGraphDestroy(g); return r; }
        if (e != cudaSuccess) return fail(c, LBCAD_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        c->graph = g;
        CK(c, cudaGraphInstantiate(&c->gexec, c->graph, 0));
      }
      CK(c, cudaGraphLaunch(c->gexec, c->stream));
      c->step += c->graph_steps;
      left -= c->graph_steps;
    }
  }
  int r = launch_steps(c, left);
  // after a fused step the a6 sums of the new state are in obs_latest
  if (r == LBCAD_OK && n > 0) c->obs_valid = c->path == LBCAD_PATH_FUSED && c->observe && !c->sync_split();
  return r;
}

int lbcad_get_fields(lbcad_ctx* c, int32_t inst, uint32_t mask, void* dst, size_t bytes, int32_t dst_is_device) {
  if (!c) return LBCAD_E_INVALID_ARG;
  if (inst < 0 || inst >= (int)c->inst.size()) return fail(c, LBCAD_E_INVALID_ARG, "instance out of range");
  if (!dst || mask == 0 || (mask & ~31u)) return fail(c, LBCAD_E_INVALID_ARG, "bad dst or mask");
  const long long N = c->inst[inst].N;
  const size_t need = (size_t)ncomp_of(mask, c->q()) * N * sizeof(double);
  if (bytes < need) return fail(c, LBCAD_E_INVALID_ARG, "dst too small");
  DeviceGuard dg(c->device);
  double* target = (double*)dst;
  if (!dst_is_device) {
    int r = ensure_staging(c, need);
    if (r) return r;
    target = c->staging;
  }
  cudaError_t e = (c->prec == LBCAD_FP64)
                      ? Launch<double, false>::get_fields(desc_now<double>(c, inst), mask, target, c->stream)
                      : Launch<float, true>::get_fields(desc_now<float>(c, inst), mask, target, c->stream);
  if (e != cudaSuccess) return fail(c, LBCAD_E_CUDA, std::string("get_fields: ") + cudaGetErrorString(e));
  if (!dst_is_device) CK(c, cudaMemcpyAsync(dst, target, need, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return LBCAD_OK;
}

int lbcad_set_fields(lbcad_ctx* c, int32_t inst, uint32_t mask, const void* src, size_t bytes,
                     int32_t src_is_device) {
  if (!c) return LBCAD_E_INVALID_ARG;
  if (inst < 0 || inst >= (int)c->inst.size()) return fail(c, LBCAD_E_INVALID_ARG, "instance out of range");
  if (!src || mask == 0 || (mask & ~31u) || (mask & LBCAD_FIELD_RHO))
    return fail(c, LBCAD_E_INVALID_ARG, "bad src or mask (RHO cannot be set)");
  const long long N = c->inst[inst].N;
  const size_t need = (size_t)ncomp_of(mask, c->q()) * N * sizeof(double);
  if (bytes < need) return fail(c, LBCAD_E_INVALID_ARG, "src too small");
  DeviceGuard dg(c->device);
  const double* from = (const double*)src;
  if (!src_is_device) {
    int r = ensure_staging(c, need);
    if (r) return r;
    CK(c, cudaMemcpyAsync(c->staging, src, need, cudaMemcpyHostToDevice, c->stream));
    from = c->staging;
  }
  Inst& I = c->inst[inst];
  const int par = (int)(c->step & 1);
  cudaError_t e;
  if (c->prec == LBCAD_FP64)
    e = Launch<double, false>::set_fields(desc_now<double>(c, inst), mask, from, (double*)I.gb[par],
                                          (double*)I.qb[par], (double*)I.pb[par], (double*)I.ub[par], c->stream);
  else
    e = Launch<float, true>::set_fields(desc_now<float>(c, inst), mask, from, (float*)I.gb[par], (float*)I.qb[par],
                                        (float*)I.pb[par], (float*)I.ub[par], c->stream);
  if (e != cudaSuccess) return fail(c, LBCAD_E_CUDA, std::string("set_fields: ") + cudaGetErrorString(e));
  c->obs_valid = false;
  CK(c, cudaStreamSynchronize(c->stream));
  return LBCAD_OK;
}

int lbcad_state_bytes(lbcad_ctx* c, int32_t inst, size_t* bytes) {
  if (!c || !bytes) return LBCAD_E_INVALID_ARG;
  if (inst < 0 || inst >= (int)c->inst.size()) return fail(c, LBCAD_E_INVALID_ARG, "instance out of range");
  *bytes = (size_t)(c->q() + 9) * (size_t)c->inst[inst].N * c->elem();
  return LBCAD_OK;
}

namespace {
// Copies the current-parity state buffers of one instance to/from a contiguous buffer.
int copy_state(lbcad_ctx* c, int inst, void* ext, size_t bytes, bool ext_is_device, bool to_ext) {
  if (inst < 0 || inst >= (int)c->inst.size()) return fail(c, LBCAD_E_INVALID_ARG, "instance out of range");
  size_t need = 0;
  lbcad_state_bytes(c, inst, &need);
  if (!ext || bytes < need) return fail(c, LBCAD_E_INVALID_ARG, "state buffer missing or too small");
  DeviceGuard dg(c->device);
  Inst& I = c->inst[inst];
  const int par = (int)(c->step & 1);
  const size_t es = c->elem(), N = (size_t)I.N;
  void* parts[4] = {I.gb[par], I.qb[par], I.pb[par], I.ub[par]};
  const size_t sizes[4] = {(size_t)c->q() * N * es, 5 * N * es, N * es, 3 * N * es};
  const cudaMemcpyKind kind = to_ext ? (ext_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost)
                                     : (ext_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
  size_t off = 0;
  for (int k = 0; k < 4; ++k) {
    char* e = (char*)ext + off;
    if (to_ext) CK(c, cudaMemcpyAsync(e, parts[k], sizes[k], kind, c->stream));
    else CK(c, cudaMemcpyAsync(parts[k], e, sizes[k], kind, c->stream));
    off += sizes[k];
  }
  if (!to_ext) c->obs_valid = false;
  CK(c, cudaStreamSynchronize(c->stream));
  return LBCAD_OK;
}
}  // namespace

int lbcad_get_state(lbcad_ctx* c, int32_t inst, void* dst, size_t bytes, int32_t dst_is_device) {
  if (!c) return LBCAD_E_INVALID_ARG;
  return copy_state(c, inst, dst, bytes, dst_is_device != 0, true);
}

int lbcad_set_state(lbcad_ctx* c, int32_t inst, const void* src, size_t bytes, int32_t src_is_device) {
  if (!c) return LBCAD_E_INVALID_ARG;
  return copy_state(c, inst, const_cast<void*>(src), bytes, src_is_device != 0, false);
}

int lbcad_observables(lbcad_ctx* c, int32_t inst, lbcad_obs* out) {
  if (!c || !out) return LBCAD_E_INVALID_ARG;
  if (inst < 0 || inst >= (int)c->inst.size()) return fail(c, LBCAD_E_INVALID_ARG, "instance out of range");
  DeviceGuard dg(c->device);
  const double* src = c->obs_latest + 12 * (size_t)inst;  // summed by the fused step
  if (!c->obs_valid) {  // another path, or the state was set: a separate reduction pass
    const Inst& I = c->inst[inst];
    long long nb = ((long long)I.g.ny * I.g.nz + kObsRowsPerBlock - 1) / kObsRowsPerBlock;
    if (nb > kObsMaxBlocks) nb = kObsMaxBlocks;
    cudaError_t e = (c->prec == LBCAD_FP64)
                        ? Launch<double, false>::observables(desc_now<double>(c, inst), c->obs_partial, (int)nb,
                                                             c->obs_out, c->stream)
                        : Launch<float, true>::observables(desc_now<float>(c, inst), c->obs_partial, (int)nb,
                                                           c->obs_out, c->stream);
    if (e != cudaSuccess) return fail(c, LBCAD_E_CUDA, std::string("observables: ") + cudaGetErrorString(e));
    src = c->obs_out;
  }
  double h[12];
  CK(c, cudaMemcpyAsync(h, src, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  out->mass = h[0];
  out->sum_psi = h[1];
  for (int a = 0; a < 3; ++a) {
    out->mom[a] = h[2 + a];
    out->cm_cos[a] = h[5 + a];
    out->cm_sin[a] = h[8 + a];
  }
  out->sum_phic = h[11];
  for (double v : h)
    if (!std::isfinite(v)) return fail(c, LBCAD_E_NAN, "non-finite value in observables");
  return LBCAD_OK;
}

}  // extern "C"

namespace {

// Copies of one stored state: g (19), Q (5), psi (1), u (3) components of n sites.
template <typename T>
struct StateBuf {
  T* g;
  T* q;
  T* p;
  T* u;
};

template <typename T>
StateBuf<T> state_at(T* base, long long N) {
  return StateBuf<T>{base, base + 19 * N, base + 24 * N, base + 25 * N};
}

template <typename T>
InstDesc<T> desc_for(const Inst& I, const StateBuf<T>& in, const StateBuf<T>& out, T* sig, T* mu, T* H) {
  InstDesc<T> d = make_desc<T>(I, 0);
  d.blk0 = 0;
  d.g_in = in.g; d.q_in = in.q; d.psi_in = in.p; d.u_in = in.u;
  d.g_out = out.g; d.q_out = out.q; d.psi_out = out.p; d.u_out = out.u;
  d.sig = sig; d.mu = mu; d.H = H;
  return d;
}

// Periodic centroid (per-axis circular mean of phi_c) from the FP64 moments.
void centroid_of(const lbcad_obs& o, const lbcad_grid& g, double X[3]) {
  const double L[3] = {(double)g.nx, (double)g.ny, (double)g.nz};
  for (int a = 0; a < 3; ++a) {
    double ang = std::atan2(o.cm_sin[a], o.cm_cos[a]);
    if (ang < 0) ang += 2.0 * 3.14159265358979323846;
    X[a] = ang * L[a] / (2.0 * 3.14159265358979323846);
  }
}

template <typename T, bool SHIFT>
int adjoint_impl(lbcad_ctx* c, int64_t nsteps, int k, double* dzeta, double* dq0, double* dQ0, double* J_out) {
  Inst& I = c->inst[0];
  const long long N = I.N;
  const int S = (int)((nsteps + k - 1) / k);
  const size_t st = 28 * (size_t)N;  // elements of one stored state
  const size_t fs = 15 * (size_t)N;  // elements of one state's sigma (9), mu, H (5)
  // buffers through the context's allocator, kept for the next call
  c->adj_lam = nullptr;
  T* ck = (T*)adj_buffer(c, 0, (size_t)S * st * sizeof(T));
  T* seg = (T*)adj_buffer(c, 1, (size_t)k * st * sizeof(T));
  T* lam = (T*)adj_buffer(c, 2, 2 * st * sizeof(T));
  T* work = (T*)adj_buffer(c, 3, (88 + 36 + 15) * (size_t)N * sizeof(T));
  T* fl = (T*)adj_buffer(c, 4, (size_t)k * fs * sizeof(T));
  const int nb = LaunchAdj<T, SHIFT>::blocks(N);
  double* pg = (double*)adj_buffer(c, 5, (2 * (size_t)nb + 2) * sizeof(double));
  InstDesc<T>* dd = (InstDesc<T>*)adj_buffer(c, 6, (size_t)k * sizeof(InstDesc<T>));
  if (!ck || !seg || !lam || !work || !fl || !pg || !dd) return fail(c, LBCAD_E_OOM, "adjoint buffers");
  T* A = work;
  T* Bf = A + 88 * N;
  T* ls = Bf + 36 * N;
  double* total = pg + 2 * nb;
  CK(c, cudaMemsetAsync(total, 0, 2 * sizeof(double), c->stream));

  lbcad_obs o0, o1;
  int r = lbcad_observables(c, 0, &o0);
  if (r) return r;
  // forward with a checkpoint at the start of every segment
  for (int sgi = 0; sgi < S; ++sgi) {
    const int par = (int)(c->step & 1);
    const StateBuf<T> cb = state_at<T>(ck + (size_t)sgi * st, N);
    CK(c, cudaMemcpyAsync(cb.g, I.gb[par], 19 * N * sizeof(T), cudaMemcpyDeviceToDevice, c->stream));
    CK(c, cudaMemcpyAsync(cb.q, I.qb[par], 5 * N * sizeof(T), cudaMemcpyDeviceToDevice, c->stream));
    CK(c, cudaMemcpyAsync(cb.p, I.pb[par], N * sizeof(T), cudaMemcpyDeviceToDevice, c->stream));
    CK(c, cudaMemcpyAsync(cb.u, I.ub[par], 3 * N * sizeof(T), cudaMemcpyDeviceToDevice, c->stream));
    const int64_t len = std::min<int64_t>(k, nsteps - (int64_t)sgi * k);
    r = lbcad_step(c, len);
    if (r) return r;
  }
  r = lbcad_observables(c, 0, &o1);
  if (r) return r;
  double X0[3], X1[3], dX[3], ks[3], kc[3];
  centroid_of(o0, I.g, X0);
  centroid_of(o1, I.g, X1);
  const double L[3] = {(double)I.g.nx, (double)I.g.ny, (double)I.g.nz};
  double J = 0.0;
  for (int a = 0; a < 3; ++a) {
    double d = X1[a] - X0[a];
    d -= L[a] * std::round(d / L[a]);  // minimum image
    dX[a] = d;
    J += 0.5 * d * d;
    const double r2 = o1.cm_cos[a] * o1.cm_cos[a] + o1.cm_sin[a] * o1.cm_sin[a];
    const double coef = (L[a] / (2.0 * 3.14159265358979323846)) / r2;
    ks[a] = coef * o1.cm_cos[a];
    kc[a] = coef * o1.cm_sin[a];
  }
  // seed: only psi at the final time enters J
  StateBuf<T> lcur = state_at<T>(lam, N), lnxt = state_at<T>(lam + st, N);
  CK(c, cudaMemsetAsync(lam, 0, st * sizeof(T), c->stream));
  cudaError_t e = LaunchAdj<T, SHIFT>::seed(desc_now<T>(c, 0), dX, ks, kc, lcur.p, c->stream);
  if (e != cudaSuccess) return fail(c, LBCAD_E_CUDA, std::string("adjoint seed: ") + cudaGetErrorString(e));

  std::vector<InstDesc<T>> hd(k);
  for (int sgi = S - 1; sgi >= 0; --sgi) {
    const int len = (int)std::min<int64_t>(k, nsteps - (int64_t)sgi * k);
    // replay the segment: states 0 .. len-1 of this segment into seg (state 0 = checkpoint)
    CK(c, cudaMemcpyAsync(seg, ck + (size_t)sgi * st, st * sizeof(T), cudaMemcpyDeviceToDevice, c->stream));
    // state j's sigma, mu, H go to its own slice of fl: the replay step that leaves state j
    // computes them, and its reverse step reads them there
    for (int j = 0; j < len; ++j) {
      const StateBuf<T> in = state_at<T>(seg + (size_t)j * st, N);
      const StateBuf<T> out = state_at<T>(seg + (size_t)(j + 1 < len ? j + 1 : j) * st, N);
      T* f = fl + (size_t)j * fs;
      hd[j] = desc_for<T>(I, in, out, f, f + 9 * N, f + 10 * N);
    }
    CK(c, cudaMemcpyAsync(dd, hd.data(), len * sizeof(InstDesc<T>), cudaMemcpyHostToDevice, c->stream));
    const long long blocks = (N + kStepBlock - 1) / kStepBlock;
    for (int j = 0; j + 1 < len; ++j) {
      e = Launch<T, SHIFT>::step(dd + j, 1, blocks, kStepBlock, c->stream);
      if (e != cudaSuccess) return fail(c, LBCAD_E_CUDA, std::string("adjoint replay: ") + cudaGetErrorString(e));
    }
    // reverse steps
    for (int j = len - 1; j >= 0; --j) {
      if (j == len - 1) {  // the segment's last state was not stepped from in the replay
        e = Launch<T, SHIFT>::fields(dd + j, 1, blocks, kStepBlock, c->stream);
        if (e != cudaSuccess) return fail(c, LBCAD_E_CUDA, std::string("adjoint fields: ") + cudaGetErrorString(e));
      }
      AdjDescHost<T> h;
      h.I = hd[j];
      h.lg = lcur.g; h.lq = lcur.q; h.lp = lcur.p; h.lu = lcur.u;
      h.A = A; h.Bf = Bf; h.ls = ls;
      h.og = lnxt.g; h.oq = lnxt.q; h.op = lnxt.p; h.ou = lnxt.u;
      h.pgrad = pg;
      e = LaunchAdj<T, SHIFT>::reverse_step(h, c->stream);
      if (e == cudaSuccess) e = adj_accumulate(pg, nb, total, c->stream);
      if (e != cudaSuccess) return fail(c, LBCAD_E_CUDA, std::string("adjoint reverse step: ") + cudaGetErrorString(e));
      std::swap(lcur, lnxt);
    }
  }
  // lcur holds the cotangent of the checkpointed initial state
  c->adj_lam = lcur.g;
  double tot[2];
  CK(c, cudaMemcpyAsync(tot, total, sizeof(tot), cudaMemcpyDeviceToHost, c->stream));
  std::vector<T> hq(5 * (size_t)N);
  CK(c, cudaMemcpyAsync(hq.data(), lcur.q, hq.size() * sizeof(T), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (dzeta) *dzeta = tot[0];
  if (dq0) *dq0 = tot[1];
  if (J_out) *J_out = J;
  if (dQ0)
    for (size_t i = 0; i < hq.size(); ++i) dQ0[i] = (double)hq[i];
  for (double v : tot)
    if (!std::isfinite(v)) return fail(c, LBCAD_E_NAN, "non-finite adjoint gradient");
  return LBCAD_OK;
}

}  // namespace

extern "C" {

int lbcad_adjoint(lbcad_ctx* c, int64_t nsteps, int32_t ckpt_every, double* dJ_dzeta, double* dJ_dq0,
                  double* dJ_dQ0, double* J) {
  if (!c) return LBCAD_E_INVALID_ARG;
  if (c->inst.size() != 1) return fail(c, LBCAD_E_UNSUPPORTED, "the adjoint runs on single-instance contexts");
  if (c->staged_only() || c->sync_split() || !c->default_lb())
    return fail(c, LBCAD_E_UNSUPPORTED, "the adjoint differentiates the Euler, lagged step of D3Q19 with the body force");
  if (nsteps < 1 || ckpt_every < 1) return fail(c, LBCAD_E_INVALID_ARG, "need nsteps >= 1 and ckpt_every >= 1");
  DeviceGuard dg(c->device);
  const int k = (int)std::min<int64_t>(ckpt_every, nsteps);
  const int r = c->prec == LBCAD_FP64 ? adjoint_impl<double, false>(c, nsteps, k, dJ_dzeta, dJ_dq0, dJ_dQ0, J)
                                      : adjoint_impl<float, true>(c, nsteps, k, dJ_dzeta, dJ_dq0, dJ_dQ0, J);
  c->obs_valid = false;  // lbcad_observables forms the sums of the final state again (separate pass)
  return r;
}

int lbcad_adjoint_fields(lbcad_ctx* c, uint32_t mask, void* dst, size_t bytes) {
  if (!c) return LBCAD_E_INVALID_ARG;
  if (!c->adj_lam) return fail(c, LBCAD_E_INVALID_ARG, "no lbcad_adjoint has run on this context");
  if (!dst || mask == 0 || (mask & ~29u)) return fail(c, LBCAD_E_INVALID_ARG, "bad dst or mask (G, U, Q, PSI)");
  const long long N = c->inst[0].N;
  const size_t need = (size_t)ncomp_of(mask) * N * sizeof(double);
  if (bytes < need) return fail(c, LBCAD_E_INVALID_ARG, "dst too small");
  DeviceGuard dg(c->device);
  int r = ensure_staging(c, need);
  if (r) return r;
  cudaError_t e = (c->prec == LBCAD_FP64)
                      ? LaunchAdj<double, false>::export_fields(desc_now<double>(c, 0), (const double*)c->adj_lam, mask,
                                                                c->staging, c->stream)
                      : LaunchAdj<float, true>::export_fields(desc_now<float>(c, 0), (const float*)c->adj_lam, mask,
                                                              c->staging, c->stream);
  if (e != cudaSuccess) return fail(c, LBCAD_E_CUDA, std::string("adjoint export: ") + cudaGetErrorString(e));
  CK(c, cudaMemcpyAsync(dst, c->staging, need, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return LBCAD_OK;
}

int lbcad_num_instances(const lbcad_ctx* c) { return c ? (int)c->inst.size() : 0; }

int lbcad_instance_grid(const lbcad_ctx* c, int32_t inst, lbcad_grid* out) {
  if (!c || !out || inst < 0 || inst >= (int)c->inst.size()) return LBCAD_E_INVALID_ARG;
  *out = c->inst[inst].g;
  return LBCAD_OK;
}

int64_t lbcad_step_count(const lbcad_ctx* c) { return c ? c->step : -1; }

void* lbcad_stream(const lbcad_ctx* c) { return c ? (void*)c->stream : nullptr; }

int lbcad_sync(lbcad_ctx* c) {
  if (!c) return LBCAD_E_INVALID_ARG;
  DeviceGuard dg(c->device);
  CK(c, cudaStreamSynchronize(c->stream));
  CK(c, cudaGetLastError());
  return LBCAD_OK;
}

void lbcad_destroy(lbcad_ctx* c) {
  if (!c) return;
  release(c);
  delete c;
}

const char* lbcad_last_error(const lbcad_ctx* c) { return c ? c->err.c_str() : g_create_err.c_str(); }

}  // extern "C"
