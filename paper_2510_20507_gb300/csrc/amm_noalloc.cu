// amm_solve_noalloc: a complete solve that allocates no device memory.
//
// Some callers cannot allocate device memory while they run: a base-station
// scheduler that computes precoders inside a per-slot deadline, where a
// cudaMalloc / cudaFree can synchronise the device and stall for far longer
// than the slot lasts, or a process that hands all device memory to its own
// pool at start-up and allows no allocation outside it.  amm_create needs
// cudaMalloc for its workspace, so those callers use this entry point: the
// workspace lives in a fixed, file-scope device array instead, and the caller
// passes only its inputs and outputs.
//
// The array (kNoAllocScratchBytes) is reserved on every GPU that loads the
// library, until the process exits.  Every call shares it and finds the
// previous call's contents there; everything a solve reads is written or
// cleared by that solve before it is read.  Calls whose work overlaps on the
// GPU (two host threads, or two streams) race on the array and must not be
// issued.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "../../include/amm.h"
#include "amm_internal.cuh"

namespace amm {

__global__ void normalize_kernel(const InstDesc* desc, const float2* Hin, const float* alpha, const float* sigma2,
                                 const float* P, float2* Hout, Scalars* sc);
__global__ void init_kernel(const InstDesc* desc, const float2* V0, const float* P, float2* V, float2* Vprev,
                            Scalars* sc, float* gamma_c, int switch_iter);
cudaError_t iterate_set_smem(int bytes);
void iterate_launch(int solves, int grid, int smem, cudaStream_t st, const IterParams& p);
amm_status check_opts(const amm_opts& o, const char** why);

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the array, looked up once per device with that device
// current (in host code the array's name is only a host-side stand-in).
// The address is cached for the life of the process: a cudaDeviceReset
// destroys the context the array lives in, after which the cached address
// is stale, so this entry point must not be used on a device after
// cudaDeviceReset has been called on it.
static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[kNoAllocMaxDevices];

static cudaError_t noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return cudaSuccess;
}

// Descriptors of a uniform batch, written on the device (no host copy).
__global__ void noalloc_desc_kernel(InstDesc* desc, int batch, InstDesc proto, long long hs, long long vs,
                                    long long us, long long cs, long long zs, long long ls) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  InstDesc D = proto;
  D.h_off = b * hs;
  D.v_off = b * vs;
  D.u_off = b * us;
  D.c_off = b * cs;
  D.z_off = b * zs;
  D.l_off = b * ls;
  desc[b] = D;
}

static size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace amm

static amm_status noalloc_fail(char* err, int err_len, amm_status s, const char* msg) {
  if (err && err_len > 0) snprintf(err, (size_t)err_len, "%s", msg);
  return s;
}

extern "C" amm_status amm_solve_noalloc(int batch, const amm_dims* dims, const amm_opts* opts, const void* H,
                                        const float* alpha, const float* sigma2, const float* P, const void* V0,
                                        int n_iters, void* V_out, double* wsr_out, void* stream, char* err,
                                        int err_len) {
  using namespace amm;
  if (err && err_len > 0) err[0] = '\0';
  if (batch < 1 || !dims || !H || !alpha || !sigma2 || !P || !V0 || !V_out || !wsr_out || n_iters < 0)
    return noalloc_fail(err, err_len, AMM_EINVAL, "amm_solve_noalloc: batch < 1, n_iters < 0 or a null pointer");
  amm_opts o;
  amm_default_opts(&o);
  if (opts) o = *opts;
  {
    // the same option checks as amm_create, then what this entry point adds
    const char* why = nullptr;
    const amm_status st = check_opts(o, &why);
    if (st != AMM_OK) {
      char msg[200];
      snprintf(msg, sizeof msg, "amm_solve_noalloc: %s", why);
      return noalloc_fail(err, err_len, st, msg);
    }
  }
  if (o.precision != AMM_FP32)
    return noalloc_fail(err, err_len, AMM_EUNSUPPORTED, "amm_solve_noalloc: only the FP32 GEMM path (AMM_FP32)");
  const amm_dims& d = dims[0];
  if (d.cells < 1 || d.cells > kMaxCells || d.users < 1 || d.nt < 1 || d.nt > 4096 || d.nr < 1 ||
      d.nr > kMaxNr || d.d < 1 || d.d > d.nr || (long long)d.cells * d.users * d.nr > 4096 ||
      (long long)d.users * d.d > 4096)
    return noalloc_fail(err, err_len, AMM_EINVAL, "amm_solve_noalloc: dims out of range");

  InstDesc proto;
  memset(&proto, 0, sizeof proto);
  proto.C = d.cells;
  proto.K = d.users;
  proto.Nt = d.nt;
  proto.Nr = d.nr;
  proto.d = d.d;
  const int budget = kSmemMax - 1024;
  const Layout Ly = plan_layout(proto, budget, o.lanczos_steps);
  if (Ly.off_H < 0 && Ly.total > budget)
    return noalloc_fail(err, err_len, AMM_EINVAL, "amm_solve_noalloc: instance too large for shared memory");
  const long long m = Ly.m, n = Ly.n, C = d.cells;
  const long long hs = C * m * d.nt, vs = C * d.nt * n, us = C * d.users, cs = C;
  // workspaces that the kernel keeps in shared memory need no scratch
  const long long zs = (Ly.off_Z < 0) ? 2 * m * Ly.ldz : 0;
  const long long ls = (Ly.off_L < 0) ? (long long)lanczos_elems(proto) : 0;

  // carve the scratch array
  size_t off = 0;
  const size_t o_desc = off;  off = up256(off + sizeof(InstDesc) * batch);
  const size_t o_sc = off;    off = up256(off + sizeof(Scalars) * batch);
  const size_t o_gc = off;    off = up256(off + sizeof(float) * cs * batch);
  const size_t o_al = off;    off = up256(off + sizeof(float) * us * batch);
  const size_t o_P = off;     off = up256(off + sizeof(float) * cs * batch);
  const size_t o_H = off;     off = up256(off + sizeof(float2) * hs * batch);
  const size_t o_Vp = off;    off = up256(off + sizeof(float2) * vs * batch);
  const size_t o_Z = off;     off = up256(off + sizeof(float2) * zs * batch);
  const size_t o_L = off;     off = up256(off + sizeof(float2) * ls * batch);
  if (off > kNoAllocScratchBytes) {
    char msg[200];
    snprintf(msg, sizeof msg,
             "amm_solve_noalloc: this batch needs %zu bytes of workspace, more than the %zu-byte static array; "
             "use a smaller batch or amm_create",
             off, kNoAllocScratchBytes);
    return noalloc_fail(err, err_len, AMM_EINVAL, msg);
  }

  void* base = nullptr;
  cudaError_t e = noalloc_scratch(&base);
  if (e != cudaSuccess) return noalloc_fail(err, err_len, AMM_ECUDA, cudaGetErrorString(e));
  unsigned char* sb = static_cast<unsigned char*>(base);
  InstDesc* desc = reinterpret_cast<InstDesc*>(sb + o_desc);
  Scalars* sc = reinterpret_cast<Scalars*>(sb + o_sc);
  float* gamma_c = reinterpret_cast<float*>(sb + o_gc);
  float* alpha_s = reinterpret_cast<float*>(sb + o_al);
  float* P_s = reinterpret_cast<float*>(sb + o_P);
  float2* Hn = reinterpret_cast<float2*>(sb + o_H);
  float2* Vprev = reinterpret_cast<float2*>(sb + o_Vp);
  float2* Zws = zs ? reinterpret_cast<float2*>(sb + o_Z) : nullptr;
  float2* Lws = ls ? reinterpret_cast<float2*>(sb + o_L) : nullptr;
  float2* V = static_cast<float2*>(V_out);
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  if ((e = iterate_set_smem(kSmemMax - 1024))) return noalloc_fail(err, err_len, AMM_ECUDA, cudaGetErrorString(e));
  // the per-instance scalars are read before the first iteration: start them at zero
  if ((e = cudaMemsetAsync(sc, 0, sizeof(Scalars) * batch, st)))
    return noalloc_fail(err, err_len, AMM_ECUDA, cudaGetErrorString(e));
  noalloc_desc_kernel<<<(batch + 255) / 256, 256, 0, st>>>(desc, batch, proto, hs, vs, us, cs, zs, ls);
  if ((e = cudaMemcpyAsync(alpha_s, alpha, sizeof(float) * us * batch, cudaMemcpyDeviceToDevice, st)) ||
      (e = cudaMemcpyAsync(P_s, P, sizeof(float) * cs * batch, cudaMemcpyDeviceToDevice, st)))
    return noalloc_fail(err, err_len, AMM_ECUDA, cudaGetErrorString(e));
  normalize_kernel<<<batch, kThreads, 0, st>>>(desc, static_cast<const float2*>(H), alpha, sigma2, P, Hn, sc);
  init_kernel<<<batch, kThreads, 0, st>>>(desc, static_cast<const float2*>(V0), P_s, V, Vprev, sc, gamma_c,
                                          o.switch_iter);
  IterParams p;
  memset(&p, 0, sizeof p);
  p.desc = desc;
  p.H = Hn;
  p.alpha = alpha_s;
  p.P = P_s;
  p.V = V;
  p.Vprev = Vprev;
  p.Zws = Zws;
  p.Lws = Lws;
  p.sc = sc;
  p.gamma_c = gamma_c;
  p.eps1 = o.eps1;
  p.eps2 = o.eps2;
  p.gamma_user = (float)o.gamma_c;
  p.tc = o.tc;
  p.extrapolate = o.extrapolate;
  p.switch_iter = o.switch_iter;
  p.step_rule = o.step_rule;
  p.lanczos_steps = o.lanczos_steps;
  p.gemm_tile = o.gemm_tile;
  p.smem_budget = budget;
  p.spin_budget = o.spin_budget > 0 ? o.spin_budget : 2000000000ll;
  if (n_iters > 0) {
    p.n_iters = n_iters;
    p.mode = kFixed;
    iterate_launch(o.fp64_solves, batch, Ly.total, st, p);
  }
  p.n_iters = 1;
  p.mode = kEvalWsr;
  p.wsr_out = wsr_out;
  iterate_launch(1, batch, Ly.total, st, p);
  if ((e = cudaGetLastError())) return noalloc_fail(err, err_len, AMM_ECUDA, cudaGetErrorString(e));
  return AMM_OK;
}
