// Plain WMMSE on the GPU (Algorithm 2, Sec. IV), one thread block per
// instance: a reference for the accelerated solver, not a fast path.
//
// Per iteration: Z = H V; per user U by eq. (9) and W = E^{-1} by eq. (10)
// (the shared FP64 solves); then for every cell k the V update of eq. (12),
//   V_k(lambda) = (A_k + lambda I)^{-1} B_k,
//   A_k = sum_r alpha_r H_{rk}^H U_r W_r U_r^H H_{rk},  B_k = [alpha_{i_k} H_{i_k k}^H U W]_i,
// with lambda = 0 when A_k is positive definite and the cell power fits, and
// otherwise bisection on [0, ||B_k||_F / sqrt(P_k)] until the interval is
// narrower than the tolerance (or the iteration cap), taking the upper end.
// Each bisection point factors A_k + lambda I by a block-wide FP32 Cholesky.
#include <math.h>

#include "amm_device.cuh"

namespace amm {

struct WLayout {
  Layout base;
  int lda;                    // leading dimension of the Nt x Nt matrices
  int off_A, off_M, off_B, off_X, off_H, off_Z, off_V;
  int total;
  bool ok;
};

__host__ __device__ inline WLayout plan_wmmse(const InstDesc& D, int budget) {
  WLayout W;
  W.base = plan_layout(D, 0, 1);
  const int m = W.base.m, Nt = D.Nt;
  W.lda = pad_ld(Nt);
  int off = align_up(W.base.total, 128);
  W.off_A = off; off += Nt * W.lda * 8;          // A_k
  W.off_M = off; off += Nt * W.lda * 8;          // A_k + lambda I, factored in place
  W.off_B = off; off += Nt * W.base.ldv * 8;     // B_k
  {                                              // solution (Nt x n) or the m x Nt product
    const int a = Nt * W.base.ldv, bq = m * W.lda;
    W.off_X = off; off += (a > bq ? a : bq) * 8;
  }
  const int szH = D.C * m * W.base.ldh * 8;
  const int szZ = m * W.base.ldz * 8;
  const int szV = D.C * Nt * W.base.ldv * 8;
  W.off_Z = off; off += szZ;
  W.off_V = off; off += szV;
  W.off_H = -1;
  if (off + szH <= budget) { W.off_H = off; off += szH; }
  W.total = off;
  W.ok = (W.off_V + szV <= budget);
  return W;
}

// Block-wide Cholesky of the Hermitian matrix in M (lower triangle used),
// in place: M = L L^H.  Returns false if a pivot is not positive.
__device__ bool block_cholesky(float2* M, int lda, int N, float* piv) {
  for (int j = 0; j < N; ++j) {
    if (threadIdx.x == 0) {
      const float d = M[(long long)j * lda + j].x;
      *piv = d;
      M[(long long)j * lda + j] = make_float2(d > 0.f ? sqrtf(d) : d, 0.f);
    }
    __syncthreads();
    if (!(*piv > 0.f)) return false;
    const float inv = rsqrtf(*piv);
    for (int i = j + 1 + threadIdx.x; i < N; i += blockDim.x) M[(long long)i * lda + j] = cscale(M[(long long)i * lda + j], inv);
    __syncthreads();
    // trailing update of the lower triangle: M[i][q] -= L[i][j] conj(L[q][j]), j < q <= i
    const int rem = N - j - 1;
    for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
      const int i = j + 1 + e / rem, q = j + 1 + e % rem;
      if (q <= i) {
        const float2 li = M[(long long)i * lda + j], lq = M[(long long)q * lda + j];
        float2 v = M[(long long)i * lda + q];
        v.x -= li.x * lq.x + li.y * lq.y;
        v.y -= li.y * lq.x - li.x * lq.y;
        M[(long long)i * lda + q] = v;
      }
    }
    __syncthreads();
  }
  return true;
}

// X = (L L^H)^{-1} B for n right-hand sides; one thread per column.
__device__ void block_chol_solve(const float2* L, int lda, int N, const float2* B, float2* X, int ldx, int n) {
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    for (int i = 0; i < N; ++i) {  // L y = b
      float2 s = B[(long long)i * ldx + c];
      for (int k = 0; k < i; ++k) s = csub(s, cmul(L[(long long)i * lda + k], X[(long long)k * ldx + c]));
      X[(long long)i * ldx + c] = cscale(s, 1.f / L[(long long)i * lda + i].x);
    }
    for (int i = N - 1; i >= 0; --i) {  // L^H x = y
      float2 s = X[(long long)i * ldx + c];
      for (int k = i + 1; k < N; ++k) {
        const float2 l = L[(long long)k * lda + i];
        s = csub(s, cmul(make_float2(l.x, -l.y), X[(long long)k * ldx + c]));
      }
      X[(long long)i * ldx + c] = cscale(s, 1.f / L[(long long)i * lda + i].x);
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads) wmmse_kernel(IterParams p, float bisect_tol, int bisect_max) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_fail;
  __shared__ float s_piv;

  const int b = p.order ? p.order[blockIdx.x] : (int)blockIdx.x;
  const InstDesc D = p.desc[b];
  Scalars* scg = p.sc + b;
  const int tid = threadIdx.x;
  const int C = D.C, K = D.K, Nt = D.Nt, Nr = D.Nr, d = D.d;
  const WLayout W = plan_wmmse(D, p.smem_budget);
  const Layout& Ly = W.base;
  const int m = Ly.m, n = Ly.n, ldz = Ly.ldz, ldv = Ly.ldv, lda = W.lda;

  if (tid == 0) {
    const int st = scg->status;
    s_fail = (st == kNumeric || st == kTimeout) ? st : kOk;
  }
  __syncthreads();
  if (s_fail != kOk) return;

  double* red = reinterpret_cast<double*>(smem + Ly.off_red);
  float2* sU = reinterpret_cast<float2*>(smem + Ly.off_U);
  float2* sUW = reinterpret_cast<float2*>(smem + Ly.off_UW);
  float2* sQ = reinterpret_cast<float2*>(smem + Ly.off_Q);
  double* sRho = reinterpret_cast<double*>(smem + Ly.off_rho);
  float2* sA = reinterpret_cast<float2*>(smem + W.off_A);
  float2* sM = reinterpret_cast<float2*>(smem + W.off_M);
  float2* sB = reinterpret_cast<float2*>(smem + W.off_B);
  float2* sX = reinterpret_cast<float2*>(smem + W.off_X);
  float2* sZ = reinterpret_cast<float2*>(smem + W.off_Z);
  float2* sV = reinterpret_cast<float2*>(smem + W.off_V);
  const float* alpha_u = p.alpha + D.u_off;
  const float* Pc = p.P + D.c_off;
  float2* Vg = p.V + D.v_off;
  float2* Vpg = p.Vprev + D.v_off;
  const float2* Hg = p.H + D.h_off;
  const float2* Hs;
  int ldh;
  if (W.off_H >= 0) {
    float2* sH = reinterpret_cast<float2*>(smem + W.off_H);
    for (long long e = tid; e < (long long)C * m * Nt; e += blockDim.x) {
      const long long r = e / Nt;
      sH[r * Ly.ldh + (e - r * Nt)] = Hg[e];
    }
    Hs = sH;
    ldh = Ly.ldh;
  } else {
    Hs = Hg;
    ldh = Nt;
  }
  for (long long e = tid; e < (long long)C * Nt * n; e += blockDim.x) {
    const long long r = e / n;
    sV[r * ldv + (e - r * n)] = Vg[e];
  }
  __syncthreads();

  for (int it = 0; it < p.n_iters; ++it) {
    // Z = H V
    for (int j = 0; j < C; ++j) {
      float2* Zo = sZ + j * n;
      block_cgemm<4, 4, 0>(m, n, Nt, Hs + (long long)j * m * ldh, ldh, sV + (long long)j * Nt * ldv, ldv,
                           [&](int r, int c, float2 v) { Zo[(long long)r * ldz + c] = v; });
    }
    __syncthreads();
    covariance_phase(D, Ly, [&](int row, int c) { return sZ[(long long)row * ldz + c]; }, sQ);
    __syncthreads();
    solve_phase<double>(D, Ly, sZ, ldz, sQ, sU, sUW, sRho, alpha_u, true, true, red, &s_fail);
    if (s_fail != kOk) break;
    const double rho = rho_sum_exact(sRho, alpha_u, Ly.CK, red);
    // V update per cell, eq. (12)
    for (int k = 0; k < C; ++k) {
      const float2* Hk = Hs + (long long)k * m * ldh;
      // T = D' H_k (m x Nt, in X), D'_r = alpha_r (U W)_r U_r^H
      for (int e = tid; e < m * Nt; e += blockDim.x) {
        const int i = e / Nt, q = e - i * Nt;
        const int r = i / Nr, a = i - r * Nr;
        const float2* Pr = sUW + r * Nr * d;
        const float2* Ur = sU + r * Nr * d;
        float2 acc = make_float2(0.f, 0.f);
        for (int s = 0; s < d; ++s) {
          float2 ts = make_float2(0.f, 0.f);  // (U_r^H H_rk)[s][q]
          for (int bb = 0; bb < Nr; ++bb) ts = cjfma(Ur[bb * d + s], Hk[(long long)(r * Nr + bb) * ldh + q], ts);
          acc = cfma(Pr[a * d + s], ts, acc);
        }
        sX[(long long)i * lda + q] = cscale(acc, alpha_u[r]);
      }
      __syncthreads();
      // A_k = H_k^H T
      block_cgemm<4, 4, 1>(Nt, Nt, m, Hk, ldh, sX, lda,
                           [&](int r, int c, float2 v) { sA[(long long)r * lda + c] = v; });
      // B_k[:, i d + s] = alpha H_{i_k k}^H (U W)_{i_k}[:, s]
      for (int e = tid; e < Nt * n; e += blockDim.x) {
        const int q = e / n, c = e - q * n;
        const int i = c / d, s = c - i * d, r = k * K + i;
        const float2* Pr = sUW + r * Nr * d;
        float2 acc = make_float2(0.f, 0.f);
        for (int a = 0; a < Nr; ++a) acc = cjfma(Hk[(long long)(r * Nr + a) * ldh + q], Pr[a * d + s], acc);
        sB[(long long)q * ldv + c] = cscale(acc, alpha_u[r]);
      }
      __syncthreads();
      double bn = 0.0;
      for (int e = tid; e < Nt * n; e += blockDim.x) bn += (double)cabs2(sB[(long long)(e / n) * ldv + e % n]);
      const double bnorm2 = block_sum(bn, red);
      // power of the solution at multiplier lam; false if A + lam I is not positive definite
      auto power_at = [&](float lam, double* pw) -> bool {
        for (int e = tid; e < Nt * Nt; e += blockDim.x) {
          const int r = e / Nt, c = e - r * Nt;
          float2 v = sA[(long long)r * lda + c];
          if (r == c) v = make_float2(v.x + lam, 0.f);
          sM[(long long)r * lda + c] = v;
        }
        __syncthreads();
        const bool ok = block_cholesky(sM, lda, Nt, &s_piv);
        if (!ok) return false;
        block_chol_solve(sM, lda, Nt, sB, sX, ldv, n);
        double part = 0.0;
        for (int e = tid; e < Nt * n; e += blockDim.x) part += (double)cabs2(sX[(long long)(e / n) * ldv + e % n]);
        *pw = block_sum(part, red);
        return true;
      };
      double pw = 0.0;
      const bool pd0 = power_at(0.f, &pw);
      if (!(pd0 && pw <= (double)Pc[k])) {
        float lo = 0.f, hi = (float)(sqrt(bnorm2) / sqrt((double)Pc[k]));
        for (int bi = 0; bi < bisect_max && (hi - lo) >= bisect_tol; ++bi) {
          const float mid = 0.5f * (lo + hi);
          const bool pd = power_at(mid, &pw);
          if (!pd || pw > (double)Pc[k]) lo = mid;
          else hi = mid;
        }
        if (!power_at(hi, &pw)) {
          if (tid == 0) s_fail = kNumeric;
          __syncthreads();
          break;
        }
      }
      // V_k = X
      float2* Vk = sV + (long long)k * Nt * ldv;
      for (int e = tid; e < Nt * n; e += blockDim.x) {
        const int q = e / n, c = e - q * n;
        Vk[(long long)q * ldv + c] = sX[(long long)q * ldv + c];
      }
      __syncthreads();
    }
    if (s_fail != kOk) break;
    if (tid == 0) scg->rho_prev = rho;
    __syncthreads();
  }
  if (s_fail == kOk) {
    for (long long e = tid; e < (long long)C * Nt * n; e += blockDim.x) {
      const long long r = e / n;
      const float2 v = sV[r * ldv + (e - r * n)];
      Vpg[e] = Vg[e];
      Vg[e] = v;
    }
  }
  if (tid == 0) scg->status = s_fail;
}

int wmmse_plan_bytes(const InstDesc* desc, int batch, int budget) {
  int mx = 0;
  for (int b = 0; b < batch; ++b) {
    const WLayout W = plan_wmmse(desc[b], budget);
    if (!W.ok || W.total > budget) return -1;
    if (W.total > mx) mx = W.total;
  }
  return mx;
}

}  // namespace amm
