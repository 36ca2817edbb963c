// lbcad_noalloc.cu -- one hybrid step that allocates no device memory.
//
// Some callers cannot let a library call cudaMalloc: for example a host framework that
// owns every byte of device memory through its own pool, or a time-critical loop that
// cannot accept the device-wide synchronisation cudaMalloc/cudaFree may cause.  For them
// lbcad_step_noalloc runs the two-kernel step with its scratch (H, mu, sigma per site)
// in a fixed file-scope device array instead of a context-owned buffer.  The caller owns
// and passes every input and output buffer.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "lbcad.h"
#include "lbcad_internal.h"
#include "lbcad_validate.h"

using namespace lbcad;

namespace {

// Scratch shared by every call on a device; every GPU that loads the library holds it
// until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[LBCAD_NOALLOC_SCRATCH_BYTES];
// The one-instance launch descriptor the step kernels read.
static __device__ __align__(256) unsigned char g_noalloc_desc[512];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};
void* g_desc_addr[kMaxDevices] = {};

int reject(int code, const std::string& msg) {
  set_thread_error(msg.c_str());
  return code;
}

// Device addresses of the file-scope arrays for the current device, looked up once per
// device (host code may not use the arrays' names as device pointers).
int device_addresses(int dev, void** scratch, void** desc) {
  if (dev < 0 || dev >= kMaxDevices) return reject(LBCAD_E_INVALID_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* s = nullptr;
    void* d = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&s, g_noalloc_scratch);
    if (e != cudaSuccess) return reject(LBCAD_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    e = cudaGetSymbolAddress(&d, g_noalloc_desc);
    if (e != cudaSuccess) return reject(LBCAD_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = s;
    g_desc_addr[dev] = d;
  }
  *scratch = g_scratch_addr[dev];
  *desc = g_desc_addr[dev];
  return LBCAD_OK;
}

template <typename T>
InstDesc<T> one_desc(const lbcad_grid& g, const lbcad_params& p, const void* g_in, const void* q_in,
                     const void* psi_in, const void* u_in, void* g_out, void* q_out, void* psi_out, void* u_out,
                     unsigned char* scratch) {
  InstDesc<T> d;
  std::memset(&d, 0, sizeof(d));
  d.nx = g.nx; d.ny = g.ny; d.nz = g.nz;
  d.N = (long long)g.nx * g.ny * g.nz;
  d.blk0 = 0;
  d.nblk = (d.N + kStepBlock - 1) / kStepBlock;
  d.g_in = (const T*)g_in; d.g_out = (T*)g_out;
  d.q_in = (const T*)q_in; d.q_out = (T*)q_out;
  d.psi_in = (const T*)psi_in; d.psi_out = (T*)psi_out;
  d.u_in = (const T*)u_in; d.u_out = (T*)u_out;
  // scratch: sigma [9][N], mu [N], H [5][N], each 256-byte aligned
  const size_t part = ((size_t)d.N * sizeof(T) + 255) & ~(size_t)255;
  d.sig = (T*)scratch;
  d.mu = (T*)(scratch + 9 * part);
  d.H = (T*)(scratch + 10 * part);
  d.c.tau_inv = (T)(1.0 / p.tau);
  d.c.guo = (T)(1.0 - 0.5 / p.tau);
  d.c.rho0 = (T)p.rho0;
  d.c.A0 = (T)p.A0; d.c.chi0 = (T)p.chi0; d.c.chis = (T)p.chis; d.c.K = (T)p.K; d.c.q0 = (T)p.q0;
  d.c.gammaQ = (T)p.gammaQ; d.c.xi = (T)p.xi; d.c.a = (T)p.a; d.c.b = (T)p.b; d.c.kphi = (T)p.kphi;
  d.c.M = (T)p.M; d.c.W = (T)p.W; d.c.zeta = (T)p.zeta;
  return d;
}

// Writes the launch descriptor into the file-scope slot.  The descriptor travels as a kernel
// argument, so nothing is read from host memory once the launch is enqueued.
template <typename T>
__global__ void k_noalloc_set_desc(InstDesc<T> d) {
  *reinterpret_cast<InstDesc<T>*>(g_noalloc_desc) = d;
}

template <typename T, bool SHIFT>
int run(const lbcad_grid& g, const lbcad_params& p, const void* g_in, const void* q_in, const void* psi_in,
        const void* u_in, void* g_out, void* q_out, void* psi_out, void* u_out, void* scratch, void* desc_dev) {
  static_assert(sizeof(InstDesc<T>) <= 512, "descriptor slot too small");
  const InstDesc<T> d = one_desc<T>(g, p, g_in, q_in, psi_in, u_in, g_out, q_out, psi_out, u_out,
                                    (unsigned char*)scratch);
  cudaStream_t s = (cudaStream_t)p.stream;
  k_noalloc_set_desc<T><<<1, 1, 0, s>>>(d);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return reject(LBCAD_E_CUDA, std::string("descriptor launch: ") + cudaGetErrorString(e));
  e = Launch<T, SHIFT>::step((const InstDesc<T>*)desc_dev, 1, d.nblk, kStepBlock, s);
  if (e != cudaSuccess) return reject(LBCAD_E_CUDA, std::string("step launch: ") + cudaGetErrorString(e));
  return LBCAD_OK;
}

}  // namespace

extern "C" int lbcad_step_noalloc(const lbcad_grid* grid, const lbcad_params* params, const void* g_in,
                                  const void* q_in, const void* psi_in, const void* u_in, void* g_out,
                                  void* q_out, void* psi_out, void* u_out) {
  set_thread_error("");
  if (!grid || !params) return reject(LBCAD_E_INVALID_ARG, "grid and params are required");
  const lbcad_grid& g = *grid;
  const lbcad_params& p = *params;
  // every host-side check comes before the buffer pointers are looked at, and none touches a device
  const std::string bad = validate(g, p);
  if (!bad.empty()) return reject(LBCAD_E_INVALID_ARG, bad);
  if (p.integrator != LBCAD_EULER || p.coupling != LBCAD_LAGGED)
    return reject(LBCAD_E_UNSUPPORTED, "only the Euler integrator with lagged coupling");
  if (p.lattice != LBCAD_D3Q19 || p.lb_form != LBCAD_LB_BODY_FORCE || p.stencil != LBCAD_STENCIL_ISO)
    return reject(LBCAD_E_UNSUPPORTED, "only D3Q19 populations, the stress as a body force, isotropic stencils");
  const size_t es = p.precision == LBCAD_FP64 ? sizeof(double) : sizeof(float);
  const long long N = (long long)g.nx * g.ny * g.nz;
  const size_t part = ((size_t)N * es + 255) & ~(size_t)255;
  if (15 * part > (size_t)LBCAD_NOALLOC_SCRATCH_BYTES)
    return reject(LBCAD_E_INVALID_ARG,
                  "grid too large for lbcad_step_noalloc: needs " + std::to_string(15 * part) +
                      " bytes of scratch, the static limit is " + std::to_string((size_t)LBCAD_NOALLOC_SCRATCH_BYTES));
  if (!g_in || !q_in || !psi_in || !u_in || !g_out || !q_out || !psi_out || !u_out)
    return reject(LBCAD_E_INVALID_ARG, "every input and output pointer is required");
  int dev = p.device;
  if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return reject(LBCAD_E_CUDA, "no CUDA device");
  int prev = -1;
  cudaGetDevice(&prev);
  if (dev != prev && cudaSetDevice(dev) != cudaSuccess) return reject(LBCAD_E_CUDA, "cudaSetDevice failed");
  void* scratch = nullptr;
  void* desc = nullptr;
  int r = device_addresses(dev, &scratch, &desc);
  if (r == LBCAD_OK)
    r = (p.precision == LBCAD_FP64)
            ? run<double, false>(g, p, g_in, q_in, psi_in, u_in, g_out, q_out, psi_out, u_out, scratch, desc)
            : run<float, true>(g, p, g_in, q_in, psi_in, u_in, g_out, q_out, psi_out, u_out, scratch, desc);
  if (prev >= 0 && prev != dev) cudaSetDevice(prev);
  return r;
}
