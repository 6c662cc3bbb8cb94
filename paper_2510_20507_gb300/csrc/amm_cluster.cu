// Multi-cell A-MMMSE iteration kernel: one thread-block cluster per
// instance, one block per cell (arXiv 2510.20507, Sec. II system model:
// every user hears every base station, so the receive covariance of eq. (9)
// couples all cells, while the gradient of eq. (14) and the projection of
// eq. (15) of cell j need only that cell's channel block).
//
// Block j of the cluster (its rank) keeps, for the whole launch, in shared
// memory: the channel block Htilde_j (the rows of every user seen from BS j,
// m = C K Nr rows by Nt), the iterate V_j^{t-1} and its column block
// Z_j = Htilde_j V_j of Z (which the gradient right-hand side Y_j overwrites
// once the extrapolation has read it).  Z(V^{t-2})_j and V_j^{t-2} stay in
// global memory (one read and one write of each per iteration, served by
// L2).  Per iteration t:
//   S3a  every block sums, for every user, its columns' part of
//        sum z z^H (compensated, about twice FP32 precision);
//   --   exchange 1: the block of user r's cell adds the C parts (distributed
//        shared memory) to Q_r, then solves its own users (eqs. (9), (10),
//        the rates) and its part of rho;
//   --   exchange 2: every block gathers U, U W of all users and the rho
//        parts (summed in rank order, so every block takes the same stage
//        and stopping decisions of Algorithm 3);
//   S6   Y_j for all users over block j's columns; S5 gamma_j by Lanczos on
//        F_j = Htilde_j^H D Htilde_j; S7 G_j = Htilde_j^H Y_j, the step, the
//        projection of cell j; Z_j = Htilde_j V_j^t for the next iteration.
// The exchanges are rounds of a cluster barrier built from one mbarrier per
// block (every block arrives on every block's barrier, release / acquire at
// cluster scope), whose waits are bounded by spin_budget: a round that runs
// out sets AMM_ETIMEOUT and ends the iterations.  A hardware cluster barrier
// at the start (all barriers initialised) and at the end (no block leaves
// while another may still read its shared memory) completes because every
// wait in between is bounded.
#include <cooperative_groups.h>
#include <math.h>

#include "amm_device.cuh"

namespace amm {
namespace cg = cooperative_groups;

constexpr int kMaxClusterCells = 8;  // portable cluster size

struct ClusterLayout {
  Layout base;  // the per-user region for all users of the instance (offsets of the plain plan)
  int ldzl;     // row stride of the local Z block
  int off_Zo, off_part, off_x, off_H, off_V, off_Z, off_L;
  int total;
  bool ok;
};

__host__ __device__ inline ClusterLayout plan_cluster(const InstDesc& D, int budget, int lanczos_steps) {
  ClusterLayout L;
  L.base = plan_layout(D, 0, lanczos_steps);  // budget 0: only the small region
  const Layout& B = L.base;
  L.ldzl = pad_ld(B.n);
  int off = align_up(B.total, 16);
  L.off_Zo = off;   off += B.CK * D.Nr * D.d * 8;   // own users' blocks of Z, compact
  off = align_up(off, 16);
  L.off_part = off; off += B.CK * B.np * 16;        // this block's covariance parts (re hi, lo, im hi, lo)
  off = align_up(off, 16);
  L.off_x = off;    off += 64;                      // exchanged scalars: rho part (ff, FP64), status
  off = align_up(off, 128);
  L.off_H = off;    off += B.m * B.ldh * 8;
  L.off_V = off;    off += D.Nt * B.ldv * 8;
  L.off_Z = off;    off += B.m * L.ldzl * 8;
  L.off_L = off;    off += lanczos_elems(D) * 8;
  L.total = off;
  L.ok = D.C >= 2 && D.C <= kMaxClusterCells && off <= budget;
  return L;
}

// One round of the cluster barrier: every thread of every block has passed
// its __syncthreads before any block leaves the round, and writes before
// the round are visible to all blocks of the cluster after it.  Returns
// false (in every thread of this block) when the wait ran past the budget.
__device__ __forceinline__ bool cluster_round(uint64_t* bar, unsigned& phase, int C, long long budget, int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("fence.acq_rel.cluster;" ::: "memory");
    const unsigned local = smem_u32(bar);
    for (int q = 0; q < C; ++q) {
      unsigned remote;
      asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(q));
      asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote) : "memory");
    }
    unsigned done = 0;
    const long long t0 = clock64();
    while (true) {
      asm volatile(
          "{\n\t.reg .pred p;\n\t"
          "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t}"
          : "=r"(done)
          : "r"(local), "r"(phase)
          : "memory");
      if (done || clock64() - t0 > budget) break;
    }
    *s_ok = (int)done;
  }
  phase ^= 1u;
  __syncthreads();
  return *s_ok != 0;
}

template <class T>
__global__ void __launch_bounds__(kThreads, 1) cluster_iterate_kernel(IterParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t mbar;  // bulk copies of this block
  __shared__ uint64_t cbar;  // cluster rounds: one arrival from every block per round
  __shared__ int s_fail, s_ok;
  __shared__ int s_ctrl[8];
  __shared__ float s_bcast;
  __shared__ ff s_rhoprev;
  __shared__ ff s_rho;
  __shared__ double s_wsr;
  __shared__ float4 s_xall[2 * kMaxClusterCells];

  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.dim_blocks().x;
  const int j = (int)cluster.block_rank();  // this block's cell
  const int inst = (int)blockIdx.x / C;
  const int b = p.order ? p.order[inst] : inst;
  const InstDesc D = p.desc[b];
  Scalars* scg = p.sc + b;
  const int tid = threadIdx.x;
  const int Nt = D.Nt, K = D.K, Nr = D.Nr, d = D.d;
  const ClusterLayout CL = plan_cluster(D, p.smem_budget, p.lanczos_steps);
  const Layout& Ly = CL.base;
  const int m = Ly.m, n = Ly.n, CK = Ly.CK, np = Ly.np, ldh = Ly.ldh, ldv = Ly.ldv, ldzl = CL.ldzl;
  const int ldz = Ly.ldz;  // row stride of the instance's global Z workspace (C n columns)

  if (tid == 0) {
    const int st = scg->status;
    s_fail = (st == kNumeric || st == kTimeout) ? st : kOk;
    if (s_fail != kOk && p.mode == kEvalWsr && j == 0) p.wsr_out[b] = __longlong_as_double(0x7ff8000000000000ll);
    s_ctrl[0] = scg->t;
    s_ctrl[1] = scg->stage;
    s_ctrl[2] = scg->stage_iter;
    s_ctrl[3] = scg->last_stage;
    s_ctrl[4] = (p.mode == kTolerance) ? 0 : scg->done;
    s_ctrl[5] = 0;
    s_rhoprev = ff_from_double(scg->rho_prev);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&cbar)), "r"(C) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (s_fail != kOk) return;  // the same status word in every block of the cluster: all return
  cluster.sync();             // every block's barrier is initialised before the first remote arrive

  double* red = reinterpret_cast<double*>(smem + Ly.off_red);
  float2* sU = reinterpret_cast<float2*>(smem + Ly.off_U);
  float2* sUW = reinterpret_cast<float2*>(smem + Ly.off_UW);
  float2* sQ = reinterpret_cast<float2*>(smem + Ly.off_Q);
  double* sRho = reinterpret_cast<double*>(smem + Ly.off_rho);
  float2* ly = reinterpret_cast<float2*>(smem + Ly.off_y);
  float2* lz = reinterpret_cast<float2*>(smem + Ly.off_z);
  float2* lD = reinterpret_cast<float2*>(smem + Ly.off_D);
  float* ta = reinterpret_cast<float*>(smem + Ly.off_tri);
  float* tb = ta + (Ly.Lm + 1);
  float* const s_alpha = reinterpret_cast<float*>(smem + Ly.off_alpha);
  float2* sZo = reinterpret_cast<float2*>(smem + CL.off_Zo);
  float4* part = reinterpret_cast<float4*>(smem + CL.off_part);
  float* xch = reinterpret_cast<float*>(smem + CL.off_x);  // [0,1] rho part (ff), [2] status, [4,5] FP64 part (lo, hi words)
  float2* sH = reinterpret_cast<float2*>(smem + CL.off_H);
  float2* sV = reinterpret_cast<float2*>(smem + CL.off_V);
  float2* sZ = reinterpret_cast<float2*>(smem + CL.off_Z);
  float2* QL = reinterpret_cast<float2*>(smem + CL.off_L);
  const float* alpha_u = s_alpha;

  for (int r = tid; r < CK; r += blockDim.x) s_alpha[r] = p.alpha[D.u_off + r];
  const float Pj = p.P[D.c_off + j];
  float* const gamma_cg = p.gamma_c + D.c_off + j;
  float gamma_c = *gamma_cg;
  float2* Vg = p.V + D.v_off + (long long)j * Nt * n;
  float2* Vpg = p.Vprev + D.v_off + (long long)j * Nt * n;
  const float2* Hg = p.H + D.h_off + (long long)j * m * Nt;
  float2* Zg = p.Zws + D.z_off;  // Z(V^{t-2}) / Y: block j is columns j n .. j n + n - 1
  const int cb = j * n;
  unsigned phase = 0, cphase = 0;

  stage_rows(sH, ldh, Hg, Nt, m, Nt, &mbar, phase, p.spin_budget, &s_fail);
  stage_rows(sV, ldv, Vg, n, Nt, n, &mbar, phase, p.spin_budget, &s_fail);
  const int tile_z = gemm_tile_for(p.gemm_tile, m, n), tile_g = gemm_tile_for(p.gemm_tile, Nt, n);
  if (p.mode != kEvalWsr && p.extrapolate && s_ctrl[0] >= 3) {  // Z(V^{t-2})_j, from V^{t-2} in global memory
    block_cgemm_tiled<0>(tile_z, m, n, Nt, sH, ldh, Vpg, n,
                         [&](int r, int c, float2 v) { Zg[(long long)r * ldz + cb + c] = v; });
  }
  block_cgemm_tiled<0>(tile_z, m, n, Nt, sH, ldh, sV, ldv, [&](int r, int c, float2 v) { sZ[r * ldzl + c] = v; });
  __syncthreads();

  const int n_iters = (p.mode == kEvalWsr) ? 1 : p.n_iters;
  ff rho = ff_from(0.f);
  for (int it = 0; it < n_iters; ++it) {
    const int t = s_ctrl[0];
    const float omega = (p.extrapolate && t >= 3) ? (float)(t - 2) / (float)(t + 1) : 0.f;
    // ---- S3a: this block's part of sum z z^H for every user (compensated
    //      sums, as in covariance_phase), and the own users' Z blocks
    for (int e = tid; e < CK * np; e += blockDim.x) {
      const int r = e / np;
      int q = e - r * np, a = 0;
      while (q >= Nr - a) {
        q -= Nr - a;
        ++a;
      }
      const int bb = a + q;
      const int own = (r / K == j) ? (r % K) * d : -1 - d;  // local own columns, if r belongs to cell j
      ff qre, qim;
      cov_entry([&](int row, int c) { return sZ[row * ldzl + c]; }, r * Nr + a, r * Nr + bb, 0, n, own, own + d,
                &qre, &qim);
      part[e] = make_float4(qre.hi, qre.lo, qim.hi, qim.lo);
    }
    for (int e = tid; e < K * Nr * d; e += blockDim.x) {
      const int i = e / (Nr * d), rem = e - i * Nr * d, a = rem / d, q = rem - a * d;
      const int r = j * K + i;
      sZo[r * Nr * d + rem] = sZ[(r * Nr + a) * ldzl + i * d + q];
    }
    // ---- exchange 1: Q_r = I + sum of the C parts, for this cell's users
    if (!cluster_round(&cbar, cphase, C, p.spin_budget, &s_ok)) {
      if (tid == 0) s_fail = kTimeout;
      break;
    }
    for (int e = tid; e < K * np; e += blockDim.x) {
      const int r = j * K + e / np, ee = e % np;
      int q = ee, a = 0;
      while (q >= Nr - a) {
        q -= Nr - a;
        ++a;
      }
      ff re = ff_from(q == 0 ? 1.f : 0.f), im = ff_from(0.f);  // q == 0: a diagonal entry
      float4 v[kMaxClusterCells];
#pragma unroll
      for (int k = 0; k < kMaxClusterCells; ++k)  // all remote loads in flight at once
        if (k < C) v[k] = cluster.map_shared_rank(part, k)[r * np + ee];
#pragma unroll
      for (int k = 0; k < kMaxClusterCells; ++k)
        if (k < C) {
          re = ff_add(re, ff_make(v[k].x, v[k].y));
          im = ff_add(im, ff_make(v[k].z, v[k].w));
        }
      sQ[r * np + ee] = make_float2(re.hi, im.hi);
      sQ[(CK + r) * np + ee] = make_float2(re.lo, im.lo);
    }
    __syncthreads();
    // ---- S3b/S4 for this cell's users
    const bool want_rate = need_rate(s_ctrl[1], p.mode, it, n_iters);
    solve_phase<T>(D, Ly, nullptr, 0, sQ, sU, sUW, sRho, alpha_u, p.mode != kEvalWsr, want_rate, red, &s_fail, sZo,
                   NoIdle(), j * K, K);
    {
      ff part_rho = ff_from(0.f);
      double part_exact = 0.0;
      for (int i = tid; i < K; i += blockDim.x) {
        const int r = j * K + i;
        if (p.mode == kEvalWsr) part_exact += (double)alpha_u[r] * sRho[r];
        else part_rho = ff_add(part_rho, ff_mul(ff_from_double(sRho[r]), ff_from(alpha_u[r])));
      }
      if (p.mode == kEvalWsr) part_exact = block_sum(part_exact, red);
      else if (want_rate) part_rho = block_sum_ff(part_rho, reinterpret_cast<float*>(red) + 80);
      else part_rho = ff_from(0.f);
      if (tid == 0) {
        xch[0] = part_rho.hi;
        xch[1] = part_rho.lo;
        xch[2] = __int_as_float(s_fail);
        xch[4] = __int_as_float(__double2loint(part_exact));
        xch[5] = __int_as_float(__double2hiint(part_exact));
      }
    }
    // ---- exchange 2: U, U W of every user; rho and the status from every block
    if (!cluster_round(&cbar, cphase, C, p.spin_budget, &s_ok)) {
      if (tid == 0) s_fail = kTimeout;
      break;
    }
    for (int e = tid; e < (C - 1) * K * Nr * d; e += blockDim.x) {
      const int kk = e / (K * Nr * d), rem = e - kk * K * Nr * d;
      const int k = kk + (kk >= j ? 1 : 0);  // every other cell
      const int off = k * K * Nr * d + rem;
      sU[off] = cluster.map_shared_rank(sU, k)[off];
      sUW[off] = cluster.map_shared_rank(sUW, k)[off];
    }
    if (tid < C) {  // one thread per rank fetches that rank's scalars
      const float4* xk = reinterpret_cast<const float4*>(cluster.map_shared_rank(xch, tid));
      s_xall[2 * tid] = xk[0];
      s_xall[2 * tid + 1] = xk[1];
    }
    __syncthreads();
    if (tid == 0) {
      ff rs = ff_from(0.f);
      double ws = 0.0;
      int f = s_fail;
      for (int k = 0; k < C; ++k) {  // rank order: the same sums in every block
        const float4 x0 = s_xall[2 * k], x1 = s_xall[2 * k + 1];
        rs = ff_add(rs, ff_make(x0.x, x0.y));
        ws += __hiloint2double(__float_as_int(x1.y), __float_as_int(x1.x));
        const int fk = __float_as_int(x0.z);
        if (fk != kOk) f = fk;
      }
      s_rho = rs;
      s_wsr = ws;
      s_fail = f;
    }
    __syncthreads();
    if (s_fail != kOk) break;
    if (p.mode == kEvalWsr) {
      if (tid == 0 && j == 0) p.wsr_out[b] = s_wsr / 0.69314718055994530942;
      break;
    }
    rho = want_rate ? s_rho : ff_from(0.f);
    if (tid == 0)
      stage_logic(s_ctrl, rho, s_rhoprev, p.mode, (float)p.eps1, (float)p.eps2, p.switch_iter, p.step_rule, p.tc);
    __syncthreads();
    if (s_ctrl[4]) break;
    const int stage = s_ctrl[1];
    const float2* sP = (stage == 2) ? sUW : sU;
    // ---- S1: Zhat = (1+w) Z(V^{t-1}) - w Z(V^{t-2}) in place in the local block, in
    //      one coalesced pass that also moves Z(V^{t-1}) to the global slot (the
    //      next iteration's Z(V^{t-2}))
    for (int e0 = 0; e0 < m * n; e0 += 8 * (int)blockDim.x) {  // eight loads in flight per thread
      float2 zp[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * blockDim.x + tid;
        if (e < m * n && omega != 0.f) {
          const int row = e / n;
          zp[u] = Zg[(long long)row * ldz + cb + (e - row * n)];
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * blockDim.x + tid;
        if (e < m * n) {
          const int row = e / n, c = e - row * n;
          const float2 zc = sZ[row * ldzl + c];
          if (omega != 0.f) sZ[row * ldzl + c] = csub(cscale(zc, 1.f + omega), cscale(zp[u], omega));
          Zg[(long long)row * ldz + cb + c] = zc;
        }
      }
    }
    __syncthreads();
    // ---- S6: Y_r over block j's columns (global numbering c), written over Zhat
    gradient_rhs_phase(
        D, Ly, [&](int row, int c) { return sZ[row * ldzl + (c - cb)]; }, sU, sP, alpha_u,
        [&](int r, int c, const float2* y) {
          for (int a = 0; a < Nr; ++a) sZ[(r * Nr + a) * ldzl + (c - cb)] = y[a];
        },
        cb, cb + n);
    __syncthreads();
    // ---- S5: gamma_j by eq. (16)
    const int sflag = s_ctrl[6];
    float gj;
    if (sflag & 1) {
      const float lam = lanczos_norm(
          D, Ly, [&](int i, int q) { return sH[i * ldh + q]; }, sU, sP, alpha_u, QL, ly, lz, lD, ta, tb, red,
          &s_bcast);
      gj = (lam > 0.f) ? 1.f / lam : 0.f;
      if (sflag & 2) gamma_c = gj;
    } else {
      gj = (p.gamma_user > 0.f) ? p.gamma_user : gamma_c;
    }
    // ---- S7: G_j = Htilde_j^H Y_j; Vtilde = Vhat - gamma G; V^{t-1} moves to the
    //      global V^{t-2} slot; ||Vtilde_j||^2 and the projection of eq. (15)
    ff nrm = ff_from(0.f);
    block_cgemm_tiled<1>(tile_g, Nt, n, m, sH, ldh, sZ, ldzl, [&](int r, int c, float2 g) {
      const float2 vc = sV[r * ldv + c];
      float2 vh = vc;
      if (omega != 0.f) vh = csub(cscale(vc, 1.f + omega), cscale(Vpg[(long long)r * n + c], omega));
      const float2 vt = csub(vh, cscale(g, gj));
      Vpg[(long long)r * n + c] = vc;
      sV[r * ldv + c] = vt;
      nrm = ff_add(nrm, ff_from(cabs2(vt)));
    });
    const ff s = block_sum_ff(nrm, reinterpret_cast<float*>(red) + 80);
    const float sj = (s.hi > Pj) ? sqrtf(Pj / s.hi) : 1.f;
    if (sj != 1.f) {
      for (int e = tid; e < Nt * n; e += blockDim.x) {
        const int r = e / n, c = e - r * n;
        sV[r * ldv + c] = cscale(sV[r * ldv + c], sj);
      }
      __syncthreads();
    }
    // ---- S2 of the next iteration: Z_j(V^t) over Y_j (consumed by the gradient GEMM)
    if (it + 1 < n_iters) {
      block_cgemm_tiled<0>(tile_z, m, n, Nt, sH, ldh, sV, ldv,
                           [&](int r, int c, float2 v) { sZ[r * ldzl + c] = v; });
    }
    __syncthreads();
    if (tid == 0) {
      s_rhoprev = rho;
      s_ctrl[3] = stage;
      s_ctrl[0] = t + 1;
      s_ctrl[5] += 1;
    }
    __syncthreads();
  }
  __syncthreads();
  if (p.mode != kEvalWsr) {
    for (int e = tid; e < Nt * n; e += blockDim.x) {
      const int r = e / n, c = e - r * n;
      Vg[e] = sV[r * ldv + c];
    }
    if (tid == 0) *gamma_cg = gamma_c;
  }
  if (tid == 0 && j == 0) {
    if (p.mode == kEvalWsr) {
      if (s_fail != kOk) {
        scg->status = s_fail;
        p.wsr_out[b] = __longlong_as_double(0x7ff8000000000000ll);
      }
    } else {
      scg->t = s_ctrl[0];
      scg->rho_prev = ff_to_double(s_rhoprev);
      scg->stage = s_ctrl[1];
      scg->stage_iter = s_ctrl[2];
      scg->last_stage = s_ctrl[3];
      int st = s_fail;
      if (p.mode == kTolerance) {
        scg->iters_run = s_ctrl[5];
        scg->done = s_ctrl[4];
        if (p.iters_out) p.iters_out[b] = s_ctrl[5];
        if (st == kOk && !s_ctrl[4]) st = kNotConv;
      }
      scg->status = st;
    }
  }
  cluster.sync();  // no block leaves while another may still read its shared memory
}

// Host side: plan, attributes and the cluster launch.
int cluster_plan_bytes(const InstDesc* desc, int batch, int budget, int lanczos_steps) {
  int mx = 0;
  for (int b = 0; b < batch; ++b) {
    const ClusterLayout L = plan_cluster(desc[b], budget, lanczos_steps);
    if (!L.ok) return -1;
    if (L.total > mx) mx = L.total;
  }
  return mx;
}

cudaError_t cluster_set_smem(int bytes) {
  cudaError_t e = cudaFuncSetAttribute(cluster_iterate_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(cluster_iterate_kernel<ff>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(cluster_iterate_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e;
}

template <class T>
static cudaLaunchConfig_t cluster_config(int batch, int C, int smem, cudaStream_t st, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(batch * C), 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// How many clusters of C blocks with this shared memory can be resident at
// once (0: the cluster does not fit this GPU).
cudaError_t cluster_max_active(int C, int smem, int* out) {
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = cluster_config<double>(1, C, smem, nullptr, attr);
  return cudaOccupancyMaxActiveClusters(out, cluster_iterate_kernel<double>, &cfg);
}

// solves: 0 FP32, 1 FP64, 2 float-float
cudaError_t cluster_launch(int solves, int batch, int C, int smem, cudaStream_t st, const IterParams& p) {
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = cluster_config<double>(batch, C, smem, st, attr);
  if (solves == 1) return cudaLaunchKernelEx(&cfg, cluster_iterate_kernel<double>, p);
  if (solves == 2) return cudaLaunchKernelEx(&cfg, cluster_iterate_kernel<ff>, p);
  return cudaLaunchKernelEx(&cfg, cluster_iterate_kernel<float>, p);
}

}  // namespace amm
