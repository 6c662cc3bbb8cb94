// C-ABI of the batched solver: context, workspace, argument checks and
// kernel launches.  See include/amm.h for the contract of each entry point.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/amm.h"
#include "amm_internal.cuh"

namespace amm {
cudaError_t iterate_set_smem(int bytes);
cudaError_t iterate_occupancy(int smem, int* per_sm);
void iterate_launch(int solves, int grid, int smem, cudaStream_t st, const IterParams& p);
__global__ void normalize_kernel(const InstDesc* desc, const float2* Hin, const float* alpha, const float* sigma2,
                                 const float* P, float2* Hout, Scalars* sc);
__global__ void init_kernel(const InstDesc* desc, const float2* V0, const float* P, float2* V, float2* Vprev,
                            Scalars* sc, float* gamma_c, int switch_iter);
cudaError_t tc_set_smem(int bytes);
void tc_launch(int solves, int grid, int smem, cudaStream_t st, const IterParams& p, int prec);
__global__ void wmmse_kernel(IterParams p, float bisect_tol, int bisect_max, int eig);
int wmmse_plan_bytes(const InstDesc* desc, int batch, int budget);
int tc_plan_bytes(const InstDesc* desc, int batch, int budget, int lanczos_steps, int prec);
int cluster_plan_bytes(const InstDesc* desc, int batch, int budget, int lanczos_steps);
cudaError_t cluster_set_smem(int bytes);
cudaError_t cluster_max_active(int C, int smem, int* out);
cudaError_t cluster_launch(int solves, int batch, int C, int smem, cudaStream_t st, const IterParams& p);

// Gather / scatter of the per-instance scalars for amm_get_state / amm_set_state.
__global__ void get_scalars_kernel(const Scalars* sc, int n, int* t, int* stage, int* stage_iter, double* rho_prev,
                                   int* status) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  if (t) t[b] = sc[b].t;
  if (stage) stage[b] = sc[b].stage;
  if (stage_iter) stage_iter[b] = sc[b].stage_iter;
  if (rho_prev) rho_prev[b] = sc[b].rho_prev;
  if (status) status[b] = sc[b].status;
}
__global__ void set_scalars_kernel(Scalars* sc, int n, const int* t, const int* stage, const int* stage_iter,
                                   const double* rho_prev) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  sc[b].t = t[b];
  sc[b].stage = stage[b];
  sc[b].stage_iter = stage_iter[b];
  sc[b].rho_prev = rho_prev[b];
  // the last iteration's stage is what a restored state continues from
  sc[b].last_stage = (t[b] > 1) ? stage[b] : 0;
  sc[b].done = 0;
}
}  // namespace amm

using amm::InstDesc;
using amm::Scalars;

struct amm_ctx {
  int batch = 0;
  int C = 0;
  amm_opts opts;
  cudaStream_t stream = nullptr;
  std::vector<InstDesc> hdesc;
  InstDesc* ddesc = nullptr;
  int* dorder = nullptr;  // block -> instance, longest first (uneven batches only)
  long long h_elems = 0, v_elems = 0, n_users = 0, n_cells = 0, z_elems = 0, l_elems = 0;
  float2* H = nullptr;
  float* alpha = nullptr;
  float* P = nullptr;
  float2* V = nullptr;
  float2* Vprev = nullptr;
  float2* Zws = nullptr;
  float2* Lws = nullptr;
  Scalars* sc = nullptr;
  float* gamma_c = nullptr;
  // device inputs of amm_solve_host, allocated on its first call
  float2* Hin = nullptr;
  float* alpha_in = nullptr;
  float* sigma2_in = nullptr;
  float* P_in = nullptr;
  float2* V0_in = nullptr;
  double* wsr_dev = nullptr;
  int smem_budget = 0;
  int smem_bytes = 0;
  int tc_bytes = 0;  // shared memory of the tensor-core kernel (0: plain path)
  int wm_bytes = 0;  // shared memory of the WMMSE kernel (-1: sizes it does not cover)
  int cl_bytes = 0;  // shared memory per block of the cluster kernel (0: not used)
  int* dqueue = nullptr;  // instance counter of the persistent schedule
  int persist_grid = 0;   // blocks of the persistent schedule (0: one block per instance)
  bool problem_set = false;
  bool started = false;
  std::string err;
  int64_t launches = 0;
};

static thread_local std::string g_create_err;

static amm_status fail(amm_ctx* ctx, amm_status s, const std::string& msg) {
  if (ctx) ctx->err = msg;
  else g_create_err = msg;
  return s;
}

static amm_status cuda_fail(amm_ctx* ctx, cudaError_t e, const char* what) {
  return fail(ctx, AMM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

static amm_status check_launch(amm_ctx* ctx, const char* what) {
  ctx->launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, what);
  return AMM_OK;
}
// the same check for a launch already counted
static amm_status check_launch_counted(amm_ctx* ctx, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, what);
  return AMM_OK;
}

extern "C" void amm_default_opts(amm_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->eps1 = 0.1;
  o->eps2 = 1e-3;
  o->tc = 3;
  o->gamma_c = 0.0;
  o->extrapolate = 1;
  o->switch_iter = -1;
  o->step_rule = 0;
  o->precision = AMM_FP32;
  o->u_at_extrapolated = 0;
  o->lanczos_steps = 64;
  o->spin_budget = 2000000000ll;  // SM clock cycles, about one second
  o->smem_budget = 0;
  o->fp64_solves = 1;
  o->gemm_tile = 0;
  o->cluster_cells = 1;
  o->schedule = 0;
}

static bool dims_ok(const amm_dims& d, std::string* why) {
  char buf[160];
  if (d.cells < 1 || d.cells > amm::kMaxCells || d.users < 1 || d.nt < 1 || d.nr < 1 || d.nr > amm::kMaxNr ||
      d.d < 1 || d.d > d.nr) {
    snprintf(buf, sizeof buf, "dims out of range: cells=%d users=%d nt=%d nr=%d d=%d", d.cells, d.users, d.nt, d.nr,
             d.d);
    *why = buf;
    return false;
  }
  const long long m = (long long)d.cells * d.users * d.nr;
  const long long n = (long long)d.users * d.d;
  if (m > 4096 || d.nt > 4096 || n > 4096) {
    snprintf(buf, sizeof buf, "instance too large: m=%lld nt=%d n=%lld (each must be <= 4096)", m, d.nt, n);
    *why = buf;
    return false;
  }
  return true;
}

// Injected allocation failures (amm_test_fail_alloc): the n-th device
// allocation from now on fails as if the device were out of memory.
static std::atomic<int> g_fail_alloc_in{0};

template <class T>
static cudaError_t dalloc(T** p, long long count) {
  *p = nullptr;
  if (count <= 0) count = 1;
  // an injected failure: counted down per allocation, fires at zero (no CUDA call)
  int left = g_fail_alloc_in.load();
  while (left > 0 && !g_fail_alloc_in.compare_exchange_weak(left, left - 1)) {
  }
  if (left == 1) return cudaErrorMemoryAllocation;
  return cudaMalloc(reinterpret_cast<void**>(p), (size_t)count * sizeof(T));
}

static void free_all(amm_ctx* c) {
  void* ptrs[] = {c->ddesc, c->dorder, c->H,     c->alpha,    c->P,         c->V,    c->Vprev,  c->Zws,   c->Lws,
                  c->sc,    c->gamma_c, c->Hin,   c->alpha_in, c->sigma2_in, c->P_in, c->V0_in, c->wsr_dev, c->dqueue};
  for (void* q : ptrs)
    if (q) cudaFree(q);
}

namespace amm {
// Option checks shared by every entry point that takes an amm_opts
// (amm_create, amm_solve_noalloc): AMM_OK, or the status and a message.
amm_status check_opts(const amm_opts& o, const char** why) {
  if (o.precision != AMM_FP32 && o.precision != AMM_BF16 && o.precision != AMM_BF16X3 && o.precision != AMM_BF16X6)
    return *why = "unknown precision", AMM_EINVAL;
  if (o.u_at_extrapolated) return *why = "u_at_extrapolated = 1 is not implemented", AMM_EUNSUPPORTED;
  if (o.step_rule < 0 || o.step_rule > 2 || o.tc < 0 || !(o.eps1 >= 0) || !(o.eps2 >= 0))
    return *why = "bad step_rule / tc / eps (step_rule in [0, 2], tc >= 0, eps1 >= 0, eps2 >= 0)", AMM_EINVAL;
  if ((o.step_rule == 2 || (o.step_rule == 0 && o.tc == 0)) && !(o.gamma_c > 0))
    return *why = "a fixed step needs gamma_c > 0", AMM_EINVAL;
  if (o.lanczos_steps < 1 || o.lanczos_steps > kMaxLanczos) return *why = "lanczos_steps must be in [1, 64]", AMM_EINVAL;
  if (o.gemm_tile < 0 || o.gemm_tile > 5) return *why = "gemm_tile must be in [0, 5]", AMM_EINVAL;
  if (o.fp64_solves < 0 || o.fp64_solves > 2) return *why = "fp64_solves must be 0, 1 or 2", AMM_EINVAL;
  if (o.schedule < 0 || o.schedule > 1) return *why = "schedule must be 0 or 1", AMM_EINVAL;
  return AMM_OK;
}
}  // namespace amm

extern "C" void amm_test_fail_alloc(int nth) { g_fail_alloc_in.store(nth > 0 ? nth : 0); }

extern "C" amm_status amm_create(amm_ctx** out, int batch, const amm_dims* dims, int n_dims, const amm_opts* opts,
                                 void* stream) {
  if (!out) return fail(nullptr, AMM_EINVAL, "out is NULL");
  *out = nullptr;
  if (batch < 1 || !dims || !(n_dims == 1 || n_dims == batch))
    return fail(nullptr, AMM_EINVAL, "need batch >= 1, dims != NULL and n_dims == 1 or batch");
  amm_opts o;
  amm_default_opts(&o);
  if (opts) o = *opts;
  {
    const char* why = nullptr;
    const amm_status st = amm::check_opts(o, &why);
    if (st != AMM_OK) return fail(nullptr, st, why);
  }
  if (o.spin_budget < 1) o.spin_budget = 2000000000ll;

  amm_ctx* c = new (std::nothrow) amm_ctx();
  if (!c) return fail(nullptr, AMM_ENOMEM, "host allocation failed");
  c->batch = batch;
  c->opts = o;
  c->stream = static_cast<cudaStream_t>(stream);
  c->hdesc.resize(batch);
  long long h = 0, v = 0, u = 0, cc = 0, z = 0, l = 0;
  int C0 = dims[0].cells;
  for (int b = 0; b < batch; ++b) {
    const amm_dims& dd = dims[n_dims == 1 ? 0 : b];
    std::string why;
    if (!dims_ok(dd, &why)) {
      delete c;
      return fail(nullptr, AMM_EINVAL, "instance " + std::to_string(b) + ": " + why);
    }
    if (dd.cells != C0) {
      delete c;
      return fail(nullptr, AMM_EINVAL, "all instances of a batch must have the same number of cells");
    }
    InstDesc& D = c->hdesc[b];
    D.C = dd.cells; D.K = dd.users; D.Nt = dd.nt; D.Nr = dd.nr; D.d = dd.d; D.pad0 = 0;
    D.h_off = h; D.v_off = v; D.u_off = u; D.c_off = cc; D.z_off = z; D.l_off = l;
    const long long m = (long long)D.C * D.K * D.Nr, n = (long long)D.K * D.d;
    h += D.C * m * D.Nt;
    v += (long long)D.C * D.Nt * n;
    u += (long long)D.C * D.K;
    cc += D.C;
    const amm::Layout Lq = amm::plan_layout(D, amm::kSmemMax, o.lanczos_steps);
    z += 2 * m * Lq.ldz;
    l += amm::lanczos_elems(D);
  }
  c->C = C0;
  c->h_elems = h; c->v_elems = v; c->n_users = u; c->n_cells = cc; c->z_elems = z; c->l_elems = l;

  // shared-memory budget: everything that fits in one block's maximum
  // (1 KB is left for the kernel's static shared variables)
  int budget = o.smem_budget;
  if (budget <= 0) budget = amm::kSmemMax - 1024;
  if (budget > amm::kSmemMax - 1024) budget = amm::kSmemMax - 1024;
  int smem = 0;
  for (int b = 0; b < batch; ++b) {
    const amm::Layout Lb = amm::plan_layout(c->hdesc[b], budget, o.lanczos_steps);
    if (Lb.off_H < 0 && Lb.total > budget) {
      delete c;
      return fail(nullptr, AMM_EINVAL, "instance " + std::to_string(b) + " needs more shared memory than available");
    }
    if (Lb.total > smem) smem = Lb.total;
  }
  c->smem_budget = budget;
  c->smem_bytes = smem;
  c->wm_bytes = amm::wmmse_plan_bytes(c->hdesc.data(), batch, budget);
  if (o.precision != AMM_FP32) {
    const int tcb = amm::tc_plan_bytes(c->hdesc.data(), batch, budget, o.lanczos_steps, o.precision);
    if (tcb < 0) {
      delete c;
      return fail(nullptr, AMM_EUNSUPPORTED,
                  "the tensor-core path needs one cell, 2*C*K*Nr <= 128, 2*Nt <= 128 and K*d <= 96");
    }
    c->tc_bytes = tcb;
  }

  cudaError_t e = cudaSuccess;
  if ((e = dalloc(&c->ddesc, batch)) || (e = dalloc(&c->H, h)) || (e = dalloc(&c->alpha, u)) ||
      (e = dalloc(&c->P, cc)) || (e = dalloc(&c->V, v)) || (e = dalloc(&c->Vprev, v)) || (e = dalloc(&c->Zws, z)) ||
      (e = dalloc(&c->Lws, l)) || (e = dalloc(&c->sc, batch)) || (e = dalloc(&c->gamma_c, cc))) {
    free_all(c);
    delete c;
    cudaGetLastError();
    return fail(nullptr, e == cudaErrorMemoryAllocation ? AMM_ENOMEM : AMM_ECUDA,
                std::string("device allocation failed: ") + cudaGetErrorString(e));
  }
  if (n_dims > 1) {
    // longest processing time first: blocks are scheduled roughly in index
    // order, so the costliest instances start first and the short ones fill in
    std::vector<double> cost(batch);
    for (int b = 0; b < batch; ++b) {
      const InstDesc& D = c->hdesc[b];
      const double m = (double)D.C * D.K * D.Nr, n = (double)D.K * D.d;
      cost[b] = 2.0 * D.C * m * D.Nt * n + 400.0 * D.C * D.K;  // GEMMs + per-user solves
    }
    std::vector<int> ord(batch);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    if ((e = dalloc(&c->dorder, batch)) ||
        (e = cudaMemcpy(c->dorder, ord.data(), sizeof(int) * batch, cudaMemcpyHostToDevice))) {
      free_all(c);
      delete c;
      return fail(nullptr, AMM_ECUDA, std::string("set-up failed: ") + cudaGetErrorString(e));
    }
  }
  if (o.precision == AMM_FP32 && o.cluster_cells && C0 >= 2) {
    // one cluster per instance where some instance's channel does not fit one block
    bool restaged = false;
    for (int b = 0; b < batch && !restaged; ++b)
      restaged = amm::plan_layout(c->hdesc[b], budget, o.lanczos_steps).off_H < 0;
    const int clb = restaged ? amm::cluster_plan_bytes(c->hdesc.data(), batch, budget, o.lanczos_steps) : -1;
    int active = 0;
    if (clb > 0 && amm::cluster_set_smem(amm::kSmemMax - 1024) == cudaSuccess &&
        amm::cluster_max_active(C0, clb, &active) == cudaSuccess && active >= 1)
      c->cl_bytes = clb;
    cudaGetLastError();  // a cluster that does not fit leaves the plain kernel in charge
  }
  if (o.schedule == 1 && c->cl_bytes == 0) {
    // persistent blocks: as many as can be resident for the plain kernel's shared memory
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) ||
        (e = amm::iterate_set_smem(amm::kSmemMax - 1024)) ||
        (e = amm::iterate_occupancy(smem, &per_sm)) || (e = dalloc(&c->dqueue, 1))) {
      free_all(c);
      delete c;
      cudaGetLastError();
      return fail(nullptr, e == cudaErrorMemoryAllocation ? AMM_ENOMEM : AMM_ECUDA,
                  std::string("persistent schedule set-up: ") + cudaGetErrorString(e));
    }
    c->persist_grid = std::min(batch, std::max(1, sms * std::max(1, per_sm)));
  }
  if ((e = cudaMemcpy(c->ddesc, c->hdesc.data(), sizeof(InstDesc) * batch, cudaMemcpyHostToDevice)) ||
      (e = cudaMemset(c->sc, 0, sizeof(Scalars) * batch)) ||
      // the limit is per kernel, not per context: raise it to the largest budget any
      // context may use so that contexts of different sizes can coexist
      (e = amm::iterate_set_smem(amm::kSmemMax - 1024)) ||
      (c->tc_bytes > 0 && (e = amm::tc_set_smem(amm::kSmemMax - 1024))) ||
      (c->wm_bytes > 0 && (e = cudaFuncSetAttribute(amm::wmmse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    amm::kSmemMax - 1024)))) {
    free_all(c);
    delete c;
    return fail(nullptr, AMM_ECUDA, std::string("set-up failed: ") + cudaGetErrorString(e));
  }
  *out = c;
  return AMM_OK;
}

extern "C" amm_status amm_sizes(const amm_ctx* c, int64_t* h, int64_t* v, int64_t* u, int64_t* cc) {
  if (!c) return AMM_EINVAL;
  if (h) *h = c->h_elems;
  if (v) *v = c->v_elems;
  if (u) *u = c->n_users;
  if (cc) *cc = c->n_cells;
  return AMM_OK;
}

extern "C" amm_status amm_set_problem(amm_ctx* c, const void* H, const float* alpha, const float* sigma2,
                                      const float* P) {
  if (!c) return AMM_EINVAL;
  if (!H || !alpha || !sigma2 || !P) return fail(c, AMM_EINVAL, "amm_set_problem: null pointer");
  amm::normalize_kernel<<<c->batch, amm::kThreads, 0, c->stream>>>(c->ddesc, static_cast<const float2*>(H), alpha,
                                                                    sigma2, P, c->H, c->sc);
  amm_status s = check_launch(c, "normalize_kernel");
  if (s) return s;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(c->alpha, alpha, sizeof(float) * c->n_users, cudaMemcpyDeviceToDevice, c->stream)) ||
      (e = cudaMemcpyAsync(c->P, P, sizeof(float) * c->n_cells, cudaMemcpyDeviceToDevice, c->stream)))
    return cuda_fail(c, e, "amm_set_problem copy");
  c->problem_set = true;
  return AMM_OK;
}

extern "C" amm_status amm_warmstart(amm_ctx* c, const void* V0) {
  if (!c) return AMM_EINVAL;
  if (!V0) return fail(c, AMM_EINVAL, "amm_warmstart: V0 is NULL");
  if (!c->problem_set) return fail(c, AMM_EINVAL, "amm_warmstart before amm_set_problem");
  amm::init_kernel<<<c->batch, amm::kThreads, 0, c->stream>>>(c->ddesc, static_cast<const float2*>(V0), c->P, c->V,
                                                               c->Vprev, c->sc, c->gamma_c, c->opts.switch_iter);
  amm_status s = check_launch(c, "init_kernel");
  if (s) return s;
  c->started = true;
  return AMM_OK;
}

static amm::IterParams base_params(amm_ctx* c) {
  amm::IterParams p;
  memset(&p, 0, sizeof p);
  p.desc = c->ddesc;
  p.order = c->dorder;
  p.H = c->H;
  p.alpha = c->alpha;
  p.P = c->P;
  p.V = c->V;
  p.Vprev = c->Vprev;
  p.Zws = c->Zws;
  p.Lws = c->Lws;
  p.sc = c->sc;
  p.gamma_c = c->gamma_c;
  p.eps1 = c->opts.eps1;
  p.eps2 = c->opts.eps2;
  p.gamma_user = (float)c->opts.gamma_c;
  p.tc = c->opts.tc;
  p.extrapolate = c->opts.extrapolate;
  p.switch_iter = c->opts.switch_iter;
  p.step_rule = c->opts.step_rule;
  p.lanczos_steps = c->opts.lanczos_steps;
  p.gemm_tile = c->opts.gemm_tile;
  p.smem_budget = c->smem_budget;
  p.spin_budget = c->opts.spin_budget;
  return p;
}

static amm_status launch_iterate(amm_ctx* c, const amm::IterParams& p) {
  // 0 FP32, 1 FP64, 2 float-float solves; the final WSR evaluation is always FP64
  const int solves = (p.mode == amm::kEvalWsr) ? 1 : c->opts.fp64_solves;
  if (c->cl_bytes > 0) {
    c->launches += 1;
    const cudaError_t e = amm::cluster_launch(solves, c->batch, c->C, c->cl_bytes, c->stream, p);
    if (e != cudaSuccess) return cuda_fail(c, e, "cluster_iterate_kernel");
    return check_launch_counted(c, "cluster_iterate_kernel");
  }
  if (c->tc_bytes > 0 && p.mode != amm::kEvalWsr) {
    amm::tc_launch(solves, c->batch, c->tc_bytes, c->stream, p, c->opts.precision);
    return check_launch(c, "tc_iterate_kernel");
  }
  if (c->persist_grid > 0 && p.mode != amm::kEvalWsr) {
    amm::IterParams q = p;
    q.queue = c->dqueue;
    q.batch = c->batch;
    const cudaError_t e = cudaMemsetAsync(c->dqueue, 0, sizeof(int), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "persistent schedule counter");
    amm::iterate_launch(solves, c->persist_grid, c->smem_bytes, c->stream, q);
    return check_launch(c, "iterate_kernel");
  }
  amm::iterate_launch(solves, c->batch, c->smem_bytes, c->stream, p);
  return check_launch(c, "iterate_kernel");
}

extern "C" amm_status amm_step(amm_ctx* c, int n_iters) {
  if (!c) return AMM_EINVAL;
  if (n_iters < 0) return fail(c, AMM_EINVAL, "amm_step: n_iters < 0");
  if (!c->started) return fail(c, AMM_EINVAL, "amm_step before amm_warmstart");
  if (n_iters == 0) return AMM_OK;
  amm::IterParams p = base_params(c);
  p.n_iters = n_iters;
  p.mode = amm::kFixed;
  return launch_iterate(c, p);
}

extern "C" amm_status amm_solve(amm_ctx* c, int max_iter, int* iters) {
  if (!c) return AMM_EINVAL;
  if (max_iter < 1) return fail(c, AMM_EINVAL, "amm_solve: max_iter < 1");
  if (!c->started) return fail(c, AMM_EINVAL, "amm_solve before amm_warmstart");
  amm::IterParams p = base_params(c);
  p.n_iters = max_iter;
  p.mode = amm::kTolerance;
  p.iters_out = iters;
  return launch_iterate(c, p);
}

extern "C" amm_status amm_wsr(amm_ctx* c, double* wsr) {
  if (!c) return AMM_EINVAL;
  if (!wsr) return fail(c, AMM_EINVAL, "amm_wsr: wsr is NULL");
  if (!c->started) return fail(c, AMM_EINVAL, "amm_wsr before amm_warmstart");
  amm::IterParams p = base_params(c);
  p.n_iters = 1;
  p.mode = amm::kEvalWsr;
  p.wsr_out = wsr;
  return launch_iterate(c, p);
}

static amm_status wmmse_launch(amm_ctx* c, const char* what, int n_iters, double bisect_tol, int bisect_max,
                               int eig) {
  if (!c) return AMM_EINVAL;
  if (n_iters < 0 || !(bisect_tol > 0) || bisect_max < 1)
    return fail(c, AMM_EINVAL, std::string(what) + ": need n_iters >= 0, bisect_tol > 0, bisect_max >= 1");
  if (!c->started) return fail(c, AMM_EINVAL, std::string(what) + " before amm_warmstart");
  if (c->wm_bytes < 0)
    return fail(c, AMM_EUNSUPPORTED, std::string(what) + ": an Nt x Nt system of these sizes does not fit shared memory");
  if (n_iters == 0) return AMM_OK;
  amm::IterParams p = base_params(c);
  p.n_iters = n_iters;
  p.mode = amm::kFixed;
  amm::wmmse_kernel<<<c->batch, amm::kThreads, c->wm_bytes, c->stream>>>(p, (float)bisect_tol, bisect_max, eig);
  return check_launch(c, "wmmse_kernel");
}

extern "C" amm_status amm_wmmse_step(amm_ctx* c, int n_iters, double bisect_tol, int bisect_max) {
  return wmmse_launch(c, "amm_wmmse_step", n_iters, bisect_tol, bisect_max, 0);
}

extern "C" amm_status amm_wmmse_step_eig(amm_ctx* c, int n_iters, double bisect_tol, int bisect_max) {
  return wmmse_launch(c, "amm_wmmse_step_eig", n_iters, bisect_tol, bisect_max, 1);
}

extern "C" amm_status amm_get_V(const amm_ctx* cc, void* V) {
  amm_ctx* c = const_cast<amm_ctx*>(cc);
  if (!c) return AMM_EINVAL;
  if (!V) return fail(c, AMM_EINVAL, "amm_get_V: V is NULL");
  cudaError_t e = cudaMemcpyAsync(V, c->V, sizeof(float2) * c->v_elems, cudaMemcpyDeviceToDevice, c->stream);
  if (e) return cuda_fail(c, e, "amm_get_V");
  return AMM_OK;
}

extern "C" amm_status amm_get_state(const amm_ctx* cc, const amm_state* st) {
  amm_ctx* c = const_cast<amm_ctx*>(cc);
  if (!c) return AMM_EINVAL;
  if (!st) return fail(c, AMM_EINVAL, "amm_get_state: st is NULL");
  cudaError_t e;
  if (st->V && (e = cudaMemcpyAsync(st->V, c->V, sizeof(float2) * c->v_elems, cudaMemcpyDeviceToDevice, c->stream)))
    return cuda_fail(c, e, "amm_get_state V");
  if (st->Vprev &&
      (e = cudaMemcpyAsync(st->Vprev, c->Vprev, sizeof(float2) * c->v_elems, cudaMemcpyDeviceToDevice, c->stream)))
    return cuda_fail(c, e, "amm_get_state Vprev");
  if (st->gamma_c &&
      (e = cudaMemcpyAsync(st->gamma_c, c->gamma_c, sizeof(float) * c->n_cells, cudaMemcpyDeviceToDevice, c->stream)))
    return cuda_fail(c, e, "amm_get_state gamma_c");
  amm::get_scalars_kernel<<<(c->batch + 255) / 256, 256, 0, c->stream>>>(c->sc, c->batch, st->t, st->stage,
                                                                          st->stage_iter, st->rho_prev, nullptr);
  return check_launch(c, "get_scalars_kernel");
}

extern "C" amm_status amm_set_state(amm_ctx* c, const amm_state* st) {
  if (!c) return AMM_EINVAL;
  if (!st || !st->V || !st->Vprev || !st->t || !st->stage || !st->stage_iter || !st->rho_prev || !st->gamma_c)
    return fail(c, AMM_EINVAL, "amm_set_state: every field is required");
  if (!c->problem_set) return fail(c, AMM_EINVAL, "amm_set_state before amm_set_problem");
  cudaError_t e;
  if ((e = cudaMemcpyAsync(c->V, st->V, sizeof(float2) * c->v_elems, cudaMemcpyDeviceToDevice, c->stream)) ||
      (e = cudaMemcpyAsync(c->Vprev, st->Vprev, sizeof(float2) * c->v_elems, cudaMemcpyDeviceToDevice, c->stream)) ||
      (e = cudaMemcpyAsync(c->gamma_c, st->gamma_c, sizeof(float) * c->n_cells, cudaMemcpyDeviceToDevice, c->stream)))
    return cuda_fail(c, e, "amm_set_state copy");
  amm::set_scalars_kernel<<<(c->batch + 255) / 256, 256, 0, c->stream>>>(c->sc, c->batch, st->t, st->stage,
                                                                          st->stage_iter, st->rho_prev);
  amm_status s = check_launch(c, "set_scalars_kernel");
  if (s) return s;
  c->started = true;
  return AMM_OK;
}

extern "C" amm_status amm_status_dev(const amm_ctx* cc, int* status) {
  amm_ctx* c = const_cast<amm_ctx*>(cc);
  if (!c) return AMM_EINVAL;
  if (!status) return fail(c, AMM_EINVAL, "amm_status_dev: status is NULL");
  amm::get_scalars_kernel<<<(c->batch + 255) / 256, 256, 0, c->stream>>>(c->sc, c->batch, nullptr, nullptr, nullptr,
                                                                          nullptr, status);
  return check_launch(c, "get_scalars_kernel");
}

extern "C" amm_status amm_solve_host(amm_ctx* c, const void* H, const float* alpha, const float* sigma2,
                                     const float* P, const void* V0, int n_iters, double* wsr_out, void* V_out) {
  if (!c) return AMM_EINVAL;
  if (!H || !alpha || !sigma2 || !P || !V0 || !wsr_out || n_iters < 0)
    return fail(c, AMM_EINVAL, "amm_solve_host: null pointer or n_iters < 0");
  cudaError_t e = cudaSuccess;
  if (!c->Hin) {
    if ((e = dalloc(&c->Hin, c->h_elems)) || (e = dalloc(&c->alpha_in, c->n_users)) ||
        (e = dalloc(&c->sigma2_in, c->n_users)) || (e = dalloc(&c->P_in, c->n_cells)) ||
        (e = dalloc(&c->V0_in, c->v_elems)) || (e = dalloc(&c->wsr_dev, c->batch))) {
      cudaGetLastError();
      return fail(c, e == cudaErrorMemoryAllocation ? AMM_ENOMEM : AMM_ECUDA,
                  std::string("amm_solve_host allocation: ") + cudaGetErrorString(e));
    }
  }
  const cudaMemcpyKind h2d = cudaMemcpyHostToDevice;
  if ((e = cudaMemcpyAsync(c->Hin, H, sizeof(float2) * c->h_elems, h2d, c->stream)) ||
      (e = cudaMemcpyAsync(c->alpha_in, alpha, sizeof(float) * c->n_users, h2d, c->stream)) ||
      (e = cudaMemcpyAsync(c->sigma2_in, sigma2, sizeof(float) * c->n_users, h2d, c->stream)) ||
      (e = cudaMemcpyAsync(c->P_in, P, sizeof(float) * c->n_cells, h2d, c->stream)) ||
      (e = cudaMemcpyAsync(c->V0_in, V0, sizeof(float2) * c->v_elems, h2d, c->stream)))
    return cuda_fail(c, e, "amm_solve_host upload");
  amm_status s;
  if ((s = amm_set_problem(c, c->Hin, c->alpha_in, c->sigma2_in, c->P_in))) return s;
  if ((s = amm_warmstart(c, c->V0_in))) return s;
  if ((s = amm_step(c, n_iters))) return s;
  if ((s = amm_wsr(c, c->wsr_dev))) return s;
  if ((e = cudaMemcpyAsync(wsr_out, c->wsr_dev, sizeof(double) * c->batch, cudaMemcpyDeviceToHost, c->stream)))
    return cuda_fail(c, e, "amm_solve_host download");
  if (V_out &&
      (e = cudaMemcpyAsync(V_out, c->V, sizeof(float2) * c->v_elems, cudaMemcpyDeviceToHost, c->stream)))
    return cuda_fail(c, e, "amm_solve_host download V");
  if ((e = cudaStreamSynchronize(c->stream))) return cuda_fail(c, e, "amm_solve_host sync");
  return AMM_OK;
}

extern "C" void amm_destroy(amm_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free_all(c);
  delete c;
}

extern "C" const char* amm_last_error(const amm_ctx* c) {
  return c ? c->err.c_str() : g_create_err.c_str();
}

extern "C" int64_t amm_launch_count(const amm_ctx* c) { return c ? c->launches : 0; }

extern "C" int amm_path(const amm_ctx* c) {
  if (!c) return -1;
  if (c->cl_bytes > 0) return 2;
  return c->tc_bytes > 0 ? 1 : 0;
}

// ---------------------------------------------------------------- CUDA graph
struct amm_graph {
  amm_ctx* ctx = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t launches = 0;  // kernel launches one replay issues
};

extern "C" amm_status amm_graph_create(amm_ctx* c, const void* H, const float* alpha, const float* sigma2,
                                       const float* P, const void* V0, int n_iters, double* wsr,
                                       amm_graph** out) {
  if (!c) return AMM_EINVAL;
  if (!out || !H || !alpha || !sigma2 || !P || !V0 || !wsr || n_iters < 1)
    return fail(c, AMM_EINVAL, "amm_graph_create: null pointer or n_iters < 1");
  *out = nullptr;
  amm_graph* g = new (std::nothrow) amm_graph();
  if (!g) return fail(c, AMM_ENOMEM, "amm_graph_create: out of host memory");
  g->ctx = c;
  cudaStream_t cap = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete g;
    return cuda_fail(c, e, "amm_graph_create: capture stream");
  }
  const cudaStream_t saved = c->stream;
  const int64_t before = c->launches;
  c->stream = cap;
  amm_status s = AMM_OK;
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    s = amm_set_problem(c, H, alpha, sigma2, P);
    if (s == AMM_OK) s = amm_warmstart(c, V0);
    if (s == AMM_OK) s = amm_step(c, n_iters);
    if (s == AMM_OK) s = amm_wsr(c, wsr);
    const cudaError_t e2 = cudaStreamEndCapture(cap, &g->graph);
    if (s == AMM_OK && e2 != cudaSuccess) s = cuda_fail(c, e2, "amm_graph_create: end capture");
  } else {
    s = cuda_fail(c, e, "amm_graph_create: begin capture");
  }
  c->stream = saved;
  cudaStreamDestroy(cap);
  g->launches = c->launches - before;
  c->launches = before;  // recorded, not launched
  if (s == AMM_OK && (e = cudaGraphInstantiate(&g->exec, g->graph, 0)) != cudaSuccess)
    s = cuda_fail(c, e, "amm_graph_create: instantiate");
  if (s != AMM_OK) {
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return s;
  }
  *out = g;
  return AMM_OK;
}

extern "C" amm_status amm_graph_launch(amm_graph* g) {
  if (!g) return AMM_EINVAL;
  const cudaError_t e = cudaGraphLaunch(g->exec, g->ctx->stream);
  if (e != cudaSuccess) return cuda_fail(g->ctx, e, "amm_graph_launch");
  g->ctx->launches += g->launches;
  return AMM_OK;
}

extern "C" void amm_graph_destroy(amm_graph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
}
