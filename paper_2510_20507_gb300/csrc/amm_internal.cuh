// Internal definitions shared by the solver's translation units: the
// per-instance descriptor, the shared-memory plan, kernel parameters and
// the complex / reduction helpers.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace amm {

constexpr int kThreads = 256;     // threads per block of every solver kernel
constexpr int kWarps = kThreads / 32;
constexpr int kMaxNr = 4;         // Nr <= 4 (small solves are unrolled for 1..4)
constexpr int kMaxCells = 16;
constexpr int kMaxLanczos = 64;
// After a wait ran past spin_budget, the kernel still waits for its own
// asynchronous copies / tensor-core operations to land, for at most this
// many SM clock cycles (about two seconds), before it moves on.
constexpr long long kDrainBudget = 4000000000ll;
constexpr int kSmemMax = 232448;  // 227 KB dynamic shared memory per block on sm_103

enum Mode { kFixed = 0, kTolerance = 1, kEvalWsr = 2 };

// Per-instance status words (values of amm_status).
enum { kOk = 0, kNumeric = 4, kTimeout = 5, kNotConv = 6 };

struct InstDesc {
  int C, K, Nt, Nr, d, pad0;
  long long h_off;  // complex elements into the channel buffer
  long long v_off;  // complex elements into V / Vprev
  long long u_off;  // users before this instance
  long long c_off;  // cells before this instance
  long long z_off;  // complex elements into the Z workspace (two m x ldz buffers)
  long long l_off;  // complex elements into the Krylov-basis workspace
};

// Iteration state of one instance, kept in device memory between launches.
struct Scalars {
  int t;           // iteration counter of Algorithm 3 (next iteration to run)
  int stage;       // 1: W = I, 2: W from eq. (10)
  int stage_iter;  // iterations run in the current stage
  int status;      // amm_status value
  double rho_prev; // R^{t-1} (nats); NaN before the first iteration
  int last_stage;  // stage of the last iteration run (0 before any)
  int iters_run;   // iterations run by the last amm_solve call
  int done;        // tolerance reached (amm_solve)
  int pad;
};

struct IterParams {
  const InstDesc* desc;
  const int* order;    // block -> instance (longest first for uneven batches); null = identity
  const float2* H;     // channels scaled by 1/sigma per user
  const float* alpha;  // per user
  const float* P;      // per cell
  float2* V;           // V^{t-1}
  float2* Vprev;       // V^{t-2}
  float2* Zws;         // Z workspace (used when Z is not resident in shared memory)
  float2* Lws;         // Krylov-basis workspace
  Scalars* sc;
  float* gamma_c;      // per cell
  double* wsr_out;     // per instance (mode kEvalWsr), bits
  int* iters_out;      // per instance (mode kTolerance), may be null
  int n_iters;
  int mode;
  double eps1, eps2;
  float gamma_user;
  int tc, extrapolate, switch_iter, step_rule, lanczos_steps, gemm_tile;
  int smem_budget;
  long long spin_budget;
  int* queue;          // non-null: persistent blocks take instances from this counter (zeroed per launch)
  int batch;           // instances of the launch (with queue)
};

// ---------------------------------------------------------------- plan
__host__ __device__ inline int pad_ld(int x) {
  int e = (x + 1) & ~1;             // even: rows are whole 16-byte units
  return (e % 4 == 0) ? e + 2 : e;  // rows shift banks by an odd number of 16-byte units
}

__host__ __device__ inline int align_up(int x, int a) { return (x + a - 1) / a * a; }

// Largest number of Krylov steps for ||F_k||_2: the option's maximum, at most
// Nt (the dimension of the space).  The iteration stops earlier once the
// largest Ritz value has settled or the Krylov space has become invariant.
// (In FP32 the space can take a step or two more than rank(F_k) + 1 to
// become numerically invariant, so the rank is no cap.)
__host__ __device__ inline int lanczos_len(const InstDesc& D, int steps) {
  int cap = D.Nt;
  if (steps < cap) cap = steps;
  if (cap > kMaxLanczos) cap = kMaxLanczos;
  return cap < 1 ? 1 : cap;
}

// Complex elements of the Lanczos vector storage: two slots of Nt.
__host__ __device__ inline int lanczos_elems(const InstDesc& D) { return 2 * D.Nt; }

// Byte offsets of the shared-memory regions of one instance.  Buffers that
// do not fit the budget live in global memory (offset -1).
struct Layout {
  int m, n, Cn, CK, np, Lm;
  int ldh, ldv, ldz;
  int off_red, off_cell, off_U, off_UW, off_Q, off_rho, off_y, off_z, off_D, off_tri, off_alpha;
  int off_H, off_Hs, off_V, off_Z, off_L, off_stage;
  int total;
};

__host__ __device__ inline Layout plan_layout(const InstDesc& D, int budget, int lanczos_steps) {
  Layout L;
  L.m = D.C * D.K * D.Nr;
  L.n = D.K * D.d;
  L.Cn = D.C * L.n;
  L.CK = D.C * D.K;
  L.np = D.Nr * (D.Nr + 1) / 2;
  L.Lm = lanczos_len(D, lanczos_steps);
  L.ldh = pad_ld(D.Nt);
  L.ldv = pad_ld(L.n);
  L.ldz = pad_ld(L.Cn);
  int off = 0;
  L.off_red = off;  off += 66 * 8;
  L.off_cell = off; off += 4 * kMaxCells * 8;
  L.off_U = off;    off += L.CK * D.Nr * D.d * 8;
  L.off_UW = off;   off += L.CK * D.Nr * D.d * 8;
  L.off_Q = off;    off += 2 * L.CK * L.np * 8;  // high parts, then low parts
  L.off_rho = off;  off += L.CK * 8;
  L.off_y = off;    off += L.m * 8;
  L.off_z = off;    off += L.m * 8;
  L.off_D = off;    off += L.CK * D.Nr * D.Nr * 8;
  L.off_tri = off;  off += 2 * (L.Lm + 1) * 4;
  off = align_up(off, 16);
  L.off_alpha = off; off += L.CK * 4;
  off = align_up(off, 128);
  const int szH = D.C * L.m * L.ldh * 8;
  const int szV = 2 * D.C * D.Nt * L.ldv * 8;
  const int szZ = 2 * L.m * L.ldz * 8;
  const int szL = lanczos_elems(D) * 8;
  // multi-cell instances whose channel does not fit get a staging buffer for
  // one cell's block Htilde_j instead (staged per GEMM from global memory)
  const int szHs = L.m * L.ldh * 8;
  // channels that stay in global memory get a staging area for the tiled
  // GEMMs (two buffers of a 64 x 16 and a 16 x 64 complex tile)
  const int szStage = 2 * (64 * 17 + 16 * 64) * 8;
  L.off_H = L.off_Hs = L.off_V = L.off_Z = L.off_L = L.off_stage = -1;
  if (off + szH <= budget) {
    L.off_H = off;
    off += szH;
  } else if (D.C > 1 && off + szHs <= budget) {
    L.off_Hs = off;
    off += szHs;
  } else if (off + szStage <= budget) {
    L.off_stage = off;
    off += szStage;
  }
  if (off + szV <= budget) { L.off_V = off; off += szV; }
  if (off + szZ <= budget) { L.off_Z = off; off += szZ; }
  if (off + szL <= budget) { L.off_L = off; off += szL; }
  L.total = off;
  return L;
}

// ---------------------------------------------------------------- complex
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// c + a*b
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
  c.x = fmaf(a.x, b.x, c.x); c.x = fmaf(-a.y, b.y, c.x);
  c.y = fmaf(a.x, b.y, c.y); c.y = fmaf(a.y, b.x, c.y);
  return c;
}
// c + conj(a)*b
__device__ __forceinline__ float2 cjfma(float2 a, float2 b, float2 c) {
  c.x = fmaf(a.x, b.x, c.x); c.x = fmaf(a.y, b.y, c.x);
  c.y = fmaf(a.x, b.y, c.y); c.y = fmaf(-a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float2 warp_sum(float2 v) {
  v.x = warp_sum(v.x);
  v.y = warp_sum(v.y);
  return v;
}

// Sum over the block in a fixed order; every thread gets the same value.
// red must hold 34 doubles.  Contains __syncthreads().
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double s = (l < kWarps) ? red[l] : 0.0;
    s = warp_sum(s);
    if (l == 0) red[33] = s;
  }
  __syncthreads();
  return red[33];
}

}  // namespace amm
