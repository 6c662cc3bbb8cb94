// Fused A-MMMSE iteration kernel (plain FP32 GEMM path), one thread block
// per instance, plus the problem-normalisation and initial-projection kernels.
//
// One iteration t of Algorithm 3 (arXiv 2510.20507, Sec. V) per loop trip:
//   S1  omega^t by eq. (18); the extrapolated point of eq. (17) is never formed
//       for the receiver: by linearity Z(Vhat) = (1+w) Z(V^{t-1}) - w Z(V^{t-2}).
//   S2  Z = H V^{t-1}: for every cell j, Z[:, cols of j] = Htilde_j V_j (complex GEMM).
//   S3  per user r: Q_r = sigma^2 I + sum over other streams of Z Z^H (the
//       interference-plus-noise covariance), then in FP64 with L = chol(Q_r),
//       X = L^{-1} Z_own, I + M = I + X^H X:
//         U_r  = T_r^{-1} Z_own = Q_r^{-1} Z_own (I+M)^{-1}      (eq. (9), Woodbury)
//         E_r  = I - U_r^H Z_own = (I+M)^{-1},  so W_r = E_r^{-1} = I + M  (eq. (10))
//         U_r W_r = Q_r^{-1} Z_own,  R_r = log det(I + M)  (the rate of Sec. II).
//   S4  rho^t = sum alpha_r R_r = WSR(V^{t-1}); the latched stage test of
//       Algorithm 3 chooses W = I (stage I) or W = E^{-1} (stage II).
//   S5  gamma_k = 1/||F_k||_2 (eq. (16)) by Lanczos on x -> Htilde_k^H D Htilde_k x
//       with D = blkdiag(2 alpha U W U^H), or the frozen gamma_c.
//   S6  Y_r = 2 alpha_r U_r W_r (U_r^H Zhat_r - S_r), S_r selecting the user's own
//       d x d identity block; then G_j = Htilde_j^H Y[:, cols of j] equals the
//       gradient (14) at Vhat exactly, without forming F_k.
//   S7  Vtilde = Vhat - gamma G, ||Vtilde_k||_F^2 (float-float accumulation), projection (15).
#include <math.h>
#include <stdio.h>

#include "amm_device.cuh"

namespace amm {

// ------------------------------------------------------------------ kernel
// All iterations of one launch for instance b, by the whole block.
template <class T>
__device__ __forceinline__ void iterate_instance(const IterParams& p, int b, unsigned char* smem, uint64_t& mbar) {
  __shared__ int s_fail;
  __shared__ int s_ctrl[8];
  __shared__ float s_bcast;
  __shared__ ff s_rhoprev;  // R^{t-1} in float-float (hi NaN: none yet)

  const InstDesc D = p.desc[b];
  Scalars* scg = p.sc + b;
  const int tid = threadIdx.x;
  const int C = D.C, Nt = D.Nt;
  const Layout Ly = plan_layout(D, p.smem_budget, p.lanczos_steps);
  const int m = Ly.m, n = Ly.n;

  if (tid == 0) {
    const int st = scg->status;
    // non-finite data, a non-PD pivot or a timed-out wait stop the instance for good;
    // "not converged" from an earlier amm_solve does not
    s_fail = (st == kNumeric || st == kTimeout) ? st : kOk;
    if (s_fail != kOk && p.mode == kEvalWsr) p.wsr_out[b] = __longlong_as_double(0x7ff8000000000000ll);
    s_ctrl[0] = scg->t;
    s_ctrl[1] = scg->stage;
    s_ctrl[2] = scg->stage_iter;
    s_ctrl[3] = scg->last_stage;
    s_ctrl[4] = (p.mode == kTolerance) ? 0 : scg->done;  // a solve call restarts its counters
    s_ctrl[5] = 0;  // iterations run by this launch
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (s_fail != kOk) return;

  double* red = reinterpret_cast<double*>(smem + Ly.off_red);
  float* cellf = reinterpret_cast<float*>(smem + Ly.off_cell);
  float2* sU = reinterpret_cast<float2*>(smem + Ly.off_U);
  float2* sUW = reinterpret_cast<float2*>(smem + Ly.off_UW);
  float2* sQ = reinterpret_cast<float2*>(smem + Ly.off_Q);
  double* sRho = reinterpret_cast<double*>(smem + Ly.off_rho);
  float2* ly = reinterpret_cast<float2*>(smem + Ly.off_y);
  float2* lz = reinterpret_cast<float2*>(smem + Ly.off_z);
  float2* lD = reinterpret_cast<float2*>(smem + Ly.off_D);
  float* ta = reinterpret_cast<float*>(smem + Ly.off_tri);
  float* tb = ta + (Ly.Lm + 1);

  // per-instance scalars live in shared memory for the whole launch:
  // cellf[32,48) P_k, [48,64) gamma_c
  float* const s_alpha = reinterpret_cast<float*>(smem + Ly.off_alpha);
  const float* alpha_u = s_alpha;
  float* gamma_cg = p.gamma_c + D.c_off;
  for (int r = tid; r < Ly.CK; r += blockDim.x) s_alpha[r] = p.alpha[D.u_off + r];
  for (int k = tid; k < C; k += blockDim.x) {
    cellf[32 + k] = p.P[D.c_off + k];
    cellf[48 + k] = gamma_cg[k];
  }
  if (tid == 0) s_rhoprev = ff_from_double(scg->rho_prev);
  const float* Pc = cellf + 32;
  float* gamma_c = cellf + 48;
  float2* Vg = p.V + D.v_off;
  float2* Vpg = p.Vprev + D.v_off;
  const float2* Hg = p.H + D.h_off;
  unsigned phase = 0;

  Views vw;
  if (Ly.off_H >= 0) {
    float2* sH = reinterpret_cast<float2*>(smem + Ly.off_H);
    stage_rows(sH, Ly.ldh, Hg, Nt, C * m, Nt, &mbar, phase, p.spin_budget, &s_fail);
    vw.H = sH;
    vw.ldh = Ly.ldh;
  } else {
    vw.H = Hg;
    vw.ldh = Nt;
  }
  const bool v_res = Ly.off_V >= 0;
  if (v_res) {
    float2* sV = reinterpret_cast<float2*>(smem + Ly.off_V);
    vw.V[0] = sV;
    vw.V[1] = sV + (long long)C * Nt * Ly.ldv;
    vw.ldv = Ly.ldv;
    stage_rows(vw.V[0], Ly.ldv, Vg, n, C * Nt, n, &mbar, phase, p.spin_budget, &s_fail);
    stage_rows(vw.V[1], Ly.ldv, Vpg, n, C * Nt, n, &mbar, phase, p.spin_budget, &s_fail);
  } else {
    vw.V[0] = Vg;
    vw.V[1] = Vpg;
    vw.ldv = n;
  }
  if (Ly.off_Z >= 0) {
    float2* sZ = reinterpret_cast<float2*>(smem + Ly.off_Z);
    vw.Z[0] = sZ;
    vw.Z[1] = sZ + (long long)m * Ly.ldz;
  } else {
    float2* Zg = p.Zws + D.z_off;
    vw.Z[0] = Zg;
    vw.Z[1] = Zg + (long long)m * Ly.ldz;
  }
  vw.ldz = Ly.ldz;
  vw.QL = (Ly.off_L >= 0) ? reinterpret_cast<float2*>(smem + Ly.off_L) : p.Lws + D.l_off;
  __syncthreads();
  if (s_fail != kOk) {
    if (tid == 0) scg->status = s_fail;
    return;
  }
  int cur = 0;  // V[cur] = V^{t-1}, V[cur^1] = V^{t-2}; Z[zc] = Z(V^{t-1}), Z[zc^1] = Z(V^{t-2})
  int zc = 0;
  const int ldv = vw.ldv, ldz = vw.ldz;
  // cell j's block Htilde_j: resident, staged into the one-cell buffer (bulk
  // copy, bounded wait) before each use, or read from global memory
  float2* sHs = (Ly.off_Hs >= 0) ? reinterpret_cast<float2*>(smem + Ly.off_Hs) : nullptr;
  const int ldh = sHs ? Ly.ldh : vw.ldh;
  auto cell_h = [&](int j) -> const float2* {
    if (!sHs) return vw.H + (long long)j * m * vw.ldh;
    __syncthreads();  // the previous user of the buffer is done
    stage_rows(sHs, Ly.ldh, Hg + (long long)j * m * Nt, Nt, m, Nt, &mbar, phase, p.spin_budget, &s_fail);
    return sHs;
  };
  const int tile_z = gemm_tile_for(p.gemm_tile, m, n), tile_g = gemm_tile_for(p.gemm_tile, Nt, n);
  // channels in global memory: the GEMMs stage their tiles through shared memory
  float2* const stage = (Ly.off_stage >= 0) ? reinterpret_cast<float2*>(smem + Ly.off_stage) : nullptr;
  auto gemm_fwd = [&](const float2* A, int lda, const float2* Bm, int ldb, auto epi) {
    if (stage) block_cgemm_staged<0>(m, n, Nt, A, lda, Bm, ldb, epi, stage);
    else block_cgemm_tiled<0>(tile_z, m, n, Nt, A, lda, Bm, ldb, epi);
  };
  auto gemm_grad = [&](const float2* A, int lda, const float2* Bm, int ldb, auto epi) {
    if (stage) block_cgemm_staged<1>(Nt, n, m, A, lda, Bm, ldb, epi, stage);
    else block_cgemm_tiled<1>(tile_g, Nt, n, m, A, lda, Bm, ldb, epi);
  };

  // Z(V^{t-2}) is needed from t = 3 on (omega > 0); rebuild it once per launch.
  if (p.mode != kEvalWsr && p.extrapolate && s_ctrl[0] >= 3) {
    for (int j = 0; j < C; ++j) {
      float2* Zo = vw.Z[zc ^ 1] + j * n;
      gemm_fwd(cell_h(j), ldh, vw.V[cur ^ 1] + (long long)j * Nt * ldv, ldv,
               [&](int r, int c, float2 v) { Zo[(long long)r * ldz + c] = v; });
    }
    __syncthreads();
  }

  // ---- S2 for the first iteration of the launch: Z = H V^{t-1}.  Every
  //      later Z = H V^t is formed per cell at the end of the previous
  //      iteration, right after that cell's V update, while its channel
  //      block is at hand (one staging of each block per iteration).
  for (int j = 0; j < C; ++j) {
    float2* Zo = vw.Z[zc] + j * n;
    gemm_fwd(cell_h(j), ldh, vw.V[cur] + (long long)j * Nt * ldv, ldv,
             [&](int r, int c, float2 v) { Zo[(long long)r * ldz + c] = v; });
  }
  __syncthreads();

  const int n_iters = (p.mode == kEvalWsr) ? 1 : p.n_iters;
  ff rho = ff_from(0.f);
  for (int it = 0; it < n_iters; ++it) {
    const int t = s_ctrl[0];
    const float omega = (p.extrapolate && t >= 3) ? (float)(t - 2) / (float)(t + 1) : 0.f;
    float2* Zc = vw.Z[zc];
    float2* Zp = vw.Z[zc ^ 1];
    // ---- S3a: interference-plus-noise covariance Q_r (upper triangle), sigma^2 = 1
    covariance_phase(D, Ly, [&](int row, int c) { return Zc[(long long)row * ldz + c]; }, sQ);
    __syncthreads();
    // ---- S3b/S4: the small solves (FP64, float-float or FP32; eight or four
    //      lanes per user); rho = WSR(V^{t-1})
    const bool want_rate = need_rate(s_ctrl[1], p.mode, it, n_iters);
    solve_phase<T>(D, Ly, Zc, ldz, sQ, sU, sUW, sRho, alpha_u, p.mode != kEvalWsr, want_rate, red, &s_fail);
    if (s_fail != kOk) break;
    if (p.mode == kEvalWsr) {
      const double w = rho_sum_exact(sRho, alpha_u, Ly.CK, red);
      if (tid == 0) p.wsr_out[b] = w / 0.69314718055994530942;
      break;
    }
    rho = want_rate ? rho_sum_ff(sRho, alpha_u, Ly.CK, red) : ff_from(0.f);
    // ---- stage test of Algorithm 3 and the stopping test (thread 0)
    if (tid == 0)
      stage_logic(s_ctrl, rho, s_rhoprev, p.mode, (float)p.eps1, (float)p.eps2, p.switch_iter, p.step_rule, p.tc);
    __syncthreads();
    if (s_ctrl[4]) break;
    const int stage = s_ctrl[1];
    const float2* sP = (stage == 2) ? sUW : sU;  // U W: W = I (stage I) or E^{-1} (stage II)
    // ---- S6: Y = 2 alpha P (U^H Zhat - S), written over Z(V^{t-2}) (each item reads its
    //      own rows of Z(V^{t-2}) before writing them)
    gradient_rhs_phase(
        D, Ly,
        [&](int row, int c) {
          const long long idx = (long long)row * ldz + c;
          float2 v = Zc[idx];
          if (omega != 0.f) v = csub(cscale(v, 1.f + omega), cscale(Zp[idx], omega));
          return v;
        },
        sU, sP, alpha_u, [&](int r, int c, const float2* y) {
          for (int a = 0; a < D.Nr; ++a) Zp[(long long)(r * D.Nr + a) * ldz + c] = y[a];
        });
    __syncthreads();
    // ---- per cell j, with its channel block staged once: S5 step size
    //      (eq. (16)), S7 G_j = Htilde_j^H Y_j, Vtilde = Vhat - gamma G over
    //      V^{t-2}, projection (eq. (15)), then Z_j = Htilde_j V_j^t for the
    //      next iteration over Y_j's columns (which G_j has consumed)
    const int sflag = s_ctrl[6];
    const bool next_z = it + 1 < n_iters;
    for (int j = 0; j < C; ++j) {
      const float2* Hj = cell_h(j);
      float gj;
      if (sflag & 1) {
        const float lam = lanczos_norm(
            D, Ly, [&](int i, int q) { return Hj[(long long)i * ldh + q]; }, sU, sP, alpha_u, vw.QL, ly, lz, lD, ta, tb,
            red, &s_bcast, Ly.off_H < 0 && !sHs);
        gj = (lam > 0.f) ? 1.f / lam : 0.f;
        if ((sflag & 2) && tid == 0) gamma_c[j] = gj;
      } else {
        gj = (p.gamma_user > 0.f) ? p.gamma_user : gamma_c[j];
      }
      const float2* Vc = vw.V[cur] + (long long)j * Nt * ldv;
      float2* Vn = vw.V[cur ^ 1] + (long long)j * Nt * ldv;
      ff nrm = ff_from(0.f);
      gemm_grad(Hj, ldh, Zp + j * n, ldz,
                           [&](int r, int c, float2 g) {
                             const long long idx = (long long)r * ldv + c;
                             float2 vh = Vc[idx];
                             if (omega != 0.f) vh = csub(cscale(vh, 1.f + omega), cscale(Vn[idx], omega));
                             const float2 vt = csub(vh, cscale(g, gj));
                             Vn[idx] = vt;
                             nrm = ff_add(nrm, ff_from(cabs2(vt)));
                           });
      // ||Vtilde_j||^2 in float-float (block-uniform; all of Vtilde_j written), then eq. (15)
      const ff s = block_sum_ff(nrm, reinterpret_cast<float*>(red) + 80);
      const float sj = (s.hi > Pc[j]) ? sqrtf(Pc[j] / s.hi) : 1.f;
      if (sj != 1.f) {
        for (int e = tid; e < Nt * n; e += blockDim.x) {
          const int r = e / n, c = e - r * n;
          Vn[(long long)r * ldv + c] = cscale(Vn[(long long)r * ldv + c], sj);
        }
        __syncthreads();
      }
      if (next_z) {
        float2* Zo = Zp + j * n;
        gemm_fwd(Hj, ldh, Vn, ldv, [&](int r, int c, float2 v) { Zo[(long long)r * ldz + c] = v; });
      }
    }
    __syncthreads();
    cur ^= 1;
    zc ^= 1;
    if (tid == 0) {
      s_rhoprev = rho;
      s_ctrl[3] = stage;
      s_ctrl[0] = t + 1;
      s_ctrl[5] += 1;
    }
    __syncthreads();
  }
  __syncthreads();
  if (p.mode == kEvalWsr) {
    if (tid == 0 && s_fail != kOk) {
      scg->status = s_fail;
      p.wsr_out[b] = __longlong_as_double(0x7ff8000000000000ll);
    }
    return;
  }
  // write back the iterate (only needed when V lives in shared memory or the buffers swapped)
  if (v_res) {
    for (int e = tid; e < C * Nt * n; e += blockDim.x) {
      const int r = e / n, c = e - r * n;
      Vg[e] = vw.V[cur][(long long)r * ldv + c];
      Vpg[e] = vw.V[cur ^ 1][(long long)r * ldv + c];
    }
  } else if (cur == 1) {
    // the roles of the two global buffers swapped: swap contents back
    for (int e = tid; e < C * Nt * n; e += blockDim.x) {
      const float2 a = Vg[e];
      Vg[e] = Vpg[e];
      Vpg[e] = a;
    }
  }
  if (tid == 0) {
    scg->t = s_ctrl[0];
    scg->rho_prev = ff_to_double(s_rhoprev);
    for (int k = 0; k < C; ++k) gamma_cg[k] = gamma_c[k];
    scg->stage = s_ctrl[1];
    scg->stage_iter = s_ctrl[2];
    scg->last_stage = s_ctrl[3];
    if (p.mode == kTolerance) {
      scg->iters_run = s_ctrl[5];
      scg->done = s_ctrl[4];
      if (p.iters_out) p.iters_out[b] = s_ctrl[5];
      if (s_fail == kOk && !s_ctrl[4]) s_fail = kNotConv;
    }
    scg->status = s_fail;
  }
}

// One block per instance (blocks in the order p.order gives: longest first
// for uneven batches), or, with p.queue, persistent blocks that take the
// next instance of that order from a device counter until none is left.
template <class T>
__global__ void __launch_bounds__(kThreads) iterate_kernel(IterParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t mbar;  // bulk-copy barrier, initialised at the start of every instance
  __shared__ int s_next;
  if (!p.queue) {
    iterate_instance<T>(p, p.order ? p.order[blockIdx.x] : (int)blockIdx.x, smem, mbar);
    return;
  }
  for (;;) {
    if (threadIdx.x == 0) s_next = atomicAdd(p.queue, 1);
    __syncthreads();
    const int k = s_next;
    __syncthreads();  // every thread has read s_next before it changes
    if (k >= p.batch) break;
    iterate_instance<T>(p, p.order ? p.order[k] : k, smem, mbar);
    __syncthreads();  // the instance's last copies have completed (its waits returned)
    if (threadIdx.x == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&mbar)) : "memory");
    __syncthreads();
  }
}

// Host-side launchers (the capi translation unit does not see the templates).
cudaError_t iterate_set_smem(int bytes) {
  cudaError_t e = cudaFuncSetAttribute(iterate_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(iterate_kernel<ff>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(iterate_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}
// Blocks of the plain kernel (FP64 solves, the largest) resident per SM with this shared memory.
cudaError_t iterate_occupancy(int smem, int* per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, iterate_kernel<double>, kThreads, (size_t)smem);
}
// solves: 0 FP32, 1 FP64, 2 float-float
void iterate_launch(int solves, int grid, int smem, cudaStream_t st, const IterParams& p) {
  if (solves == 1) iterate_kernel<double><<<grid, kThreads, smem, st>>>(p);
  else if (solves == 2) iterate_kernel<ff><<<grid, kThreads, smem, st>>>(p);
  else iterate_kernel<float><<<grid, kThreads, smem, st>>>(p);
}

// ------------------------------------------------------------------ set-up kernels
// H_j rows of user r scaled by 1/sigma_r; status per instance.
__global__ void normalize_kernel(const InstDesc* desc, const float2* Hin, const float* alpha, const float* sigma2,
                                 const float* P, float2* Hout, Scalars* sc) {
  const InstDesc D = desc[blockIdx.x];
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  const int m = D.C * D.K * D.Nr;
  const long long total = (long long)D.C * m * D.Nt;
  for (long long e = threadIdx.x; e < total; e += blockDim.x) {
    const long long row = e / D.Nt;
    const int r = (int)(row % m) / D.Nr;
    const float s2 = sigma2[D.u_off + r];
    const float2 h = Hin[D.h_off + e];
    const float sc = rsqrtf(s2);
    if (!(s2 > 0.f) || !isfinite(h.x) || !isfinite(h.y) || !isfinite(sc)) bad = 1;
    Hout[D.h_off + e] = make_float2(h.x * sc, h.y * sc);
  }
  for (int r = threadIdx.x; r < D.C * D.K; r += blockDim.x)
    if (!isfinite(alpha[D.u_off + r]) || !(alpha[D.u_off + r] >= 0.f)) bad = 1;
  for (int k = threadIdx.x; k < D.C; k += blockDim.x)
    if (!isfinite(P[D.c_off + k]) || !(P[D.c_off + k] > 0.f)) bad = 1;
  __syncthreads();
  if (threadIdx.x == 0) sc[blockIdx.x].status = bad ? kNumeric : kOk;
}

// V^0 = projection of V0 onto each cell's ball (eq. (15)); V^{-1} = V^0; reset state.
__global__ void init_kernel(const InstDesc* desc, const float2* V0, const float* P, float2* V, float2* Vprev,
                            Scalars* sc, float* gamma_c, int switch_iter) {
  const InstDesc D = desc[blockIdx.x];
  __shared__ double red[34];
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  const int blk = D.Nt * D.K * D.d;
  for (int k = 0; k < D.C; ++k) {
    const float2* src = V0 + D.v_off + (long long)k * blk;
    double part = 0.0;
    for (int e = threadIdx.x; e < blk; e += blockDim.x) {
      const float2 v = src[e];
      if (!isfinite(v.x) || !isfinite(v.y)) bad = 1;
      part += (double)v.x * v.x + (double)v.y * v.y;
    }
    const double s = block_sum(part, red);
    const double Pk = P[D.c_off + k];
    const float scale = (s > Pk) ? (float)sqrt(Pk / s) : 1.f;
    for (int e = threadIdx.x; e < blk; e += blockDim.x) {
      const float2 v = cscale(src[e], scale);
      V[D.v_off + (long long)k * blk + e] = v;
      Vprev[D.v_off + (long long)k * blk + e] = v;
    }
    if (threadIdx.x == 0) gamma_c[D.c_off + k] = 0.f;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    Scalars& s = sc[blockIdx.x];
    s.t = 1;
    s.stage = (switch_iter == 1) ? 2 : 1;
    s.stage_iter = 0;
    s.rho_prev = __longlong_as_double(0x7ff8000000000000ll);  // NaN: no R^{t-1} yet
    s.last_stage = 0;
    s.iters_run = 0;
    s.done = 0;
    if (bad && s.status == kOk) s.status = kNumeric;
  }
}

}  // namespace amm
