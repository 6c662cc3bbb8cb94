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
// Each bisection point factors A_k + lambda I by a block-wide FP32 Cholesky;
// or (eig = 1) A_k = Q diag(l) Q^H is decomposed once per cell and
// iteration by Jacobi rotations, after which every bisection point costs
// O(Nt n): ||V_k(lambda)||_F^2 = sum_i w_i / (l_i + lambda)^2 with w_i the
// squared norm of row i of Q^H B_k, and V_k = Q diag(1 / (l + lambda)) Q^H B_k.
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

// X = (L L^H)^{-1} B for n right-hand sides (B and X with row stride ldx):
// g consecutive lanes per column (g a power of two, g n <= the block), each
// step of the substitutions summing its inner product over the g lanes and
// one shuffle reduction; the lead lane writes the new entry.
__device__ void block_chol_solve(const float2* L, int lda, int N, const float2* B, float2* X, int ldx, int n) {
  int g = 1;
  while (g < 32 && 2 * g * n <= (int)blockDim.x) g <<= 1;
  const int cg = (int)threadIdx.x / g, l = (int)threadIdx.x - cg * g, ncg = (int)blockDim.x / g;
  for (int c0 = 0; c0 < n; c0 += ncg) {  // block-uniform trip count
    const int c = c0 + cg;
    const bool act = c < n;
    for (int i = 0; i < N; ++i) {  // L y = b
      float2 part = make_float2(0.f, 0.f);
      if (act)
        for (int k = l; k < i; k += g) part = cfma(L[(long long)i * lda + k], X[(long long)k * ldx + c], part);
      for (int o = g >> 1; o > 0; o >>= 1) {
        part.x += __shfl_xor_sync(0xffffffffu, part.x, o, g);
        part.y += __shfl_xor_sync(0xffffffffu, part.y, o, g);
      }
      if (act && l == 0)
        X[(long long)i * ldx + c] = cscale(csub(B[(long long)i * ldx + c], part), 1.f / L[(long long)i * lda + i].x);
      __syncwarp();
    }
    for (int i = N - 1; i >= 0; --i) {  // L^H x = y
      float2 part = make_float2(0.f, 0.f);
      if (act)
        for (int k = i + 1 + l; k < N; k += g)
          part = cjfma(L[(long long)k * lda + i], X[(long long)k * ldx + c], part);
      for (int o = g >> 1; o > 0; o >>= 1) {
        part.x += __shfl_xor_sync(0xffffffffu, part.x, o, g);
        part.y += __shfl_xor_sync(0xffffffffu, part.y, o, g);
      }
      if (act && l == 0)
        X[(long long)i * ldx + c] = cscale(csub(X[(long long)i * ldx + c], part), 1.f / L[(long long)i * lda + i].x);
      __syncwarp();
    }
  }
  __syncthreads();
}

// Index pair i of round r of a sweep over n2 (even) indices in the round-robin
// (tournament) order: index 0 stays, the others rotate, so every pair meets
// once per sweep of n2 - 1 rounds and the pairs of a round are disjoint.
__device__ __forceinline__ int2 jacobi_pair(int i, int r, int n2) {
  const int p = (i == 0) ? 0 : ((i - 1 + r) % (n2 - 1)) + 1;
  const int q = ((n2 - 2 - i + r) % (n2 - 1)) + 1;
  return make_int2(p, q);
}

// Eigen-decomposition of the Hermitian N x N matrix in A (row stride lda) by
// cyclic Jacobi rotations, block-wide, all rotations of a round at once (their
// index pairs are disjoint): per pair (p, q) with A_pq = |c| e^{i phi}, the
// unitary J = diag(1, e^{-i phi}) R, R the real rotation that diagonalises
// [[A_pp, |c|], [|c|, A_qq]] (t = sign(tau) / (|tau| + sqrt(1 + tau^2)),
// tau = (A_qq - A_pp) / (2 |c|), cos = 1 / sqrt(1 + t^2), sin = t cos);
// A <- J^H A J by a row pass then a column pass, Q <- Q J.  Sweeps until the
// off-diagonal mass is below (1e-5)^2 of ||A||_F^2 (FP32 rounding keeps it
// near (1e-6)^2, where further sweeps stall), at most max_sweeps.  On
// return the diagonal of A holds the eigenvalues (real parts) and the
// columns of Q (row stride lda) the eigenvectors.  rot: N / 2 + 1 float4 and
// as many int2 after them (the round's pairs).  Contains __syncthreads().
__device__ void block_jacobi_eig(float2* A, float2* Q, int lda, int N, float4* rot, double* red, int max_sweeps) {
  const int n2 = N + (N & 1), npair = n2 / 2;
  int2* pairs = reinterpret_cast<int2*>(rot + npair);
  double fp = 0.0;
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int r = e / N, c = e - r * N;
    Q[(long long)r * lda + c] = make_float2(r == c ? 1.f : 0.f, 0.f);
    fp += (double)cabs2(A[(long long)r * lda + c]);
  }
  const double fro = block_sum(fp, red);
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    double op = 0.0;
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
      const int r = e / N, c = e - r * N;
      if (r != c) op += (double)cabs2(A[(long long)r * lda + c]);
    }
    if (!(block_sum(op, red) > 1e-10 * fro)) break;
    for (int rr = 0; rr < n2 - 1; ++rr) {
      // the round's pairs and rotations (a pair with the padding index of an
      // odd N, or with nothing to annihilate, keeps the identity: p = -1)
      for (int i = threadIdx.x; i < npair; i += blockDim.x) {
        const int2 pq = jacobi_pair(i, rr, n2);
        float4 R = make_float4(1.f, 0.f, 1.f, 0.f);  // (cos, sin, e^{-i phi})
        int2 keep = make_int2(-1, -1);
        if (pq.x < N && pq.y < N) {
          const float a = A[(long long)pq.x * lda + pq.x].x, bq = A[(long long)pq.y * lda + pq.y].x;
          const float2 c = A[(long long)pq.x * lda + pq.y];
          const float ac = sqrtf(cabs2(c));
          if (ac > 1e-30f) {
            const float tau = (bq - a) / (2.f * ac);
            const float t = copysignf(1.f, tau) / (fabsf(tau) + sqrtf(1.f + tau * tau));
            const float cs = rsqrtf(1.f + t * t);
            R = make_float4(cs, t * cs, c.x / ac, -c.y / ac);
            keep = pq;
          }
        }
        rot[i] = R;
        pairs[i] = keep;
      }
      __syncthreads();
      // rows p, q: J^H [A_p.; A_q.] (consecutive threads: consecutive columns).
      // Four tasks per trip with every load ahead of every store: the rows of
      // different pairs never alias, which the compiler cannot see.
      for (int e0 = threadIdx.x; e0 < npair * N; e0 += 4 * blockDim.x) {
        int2 pq[4];
        int x[4];
        float4 R[4];
        float2 ap[4], aq[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int e = e0 + u * blockDim.x;
          const int i = e / N;
          x[u] = e - i * N;
          pq[u] = (e < npair * N) ? pairs[i] : make_int2(-1, -1);
          if (pq[u].x >= 0) {
            R[u] = rot[i];
            ap[u] = A[(long long)pq[u].x * lda + x[u]];
            aq[u] = A[(long long)pq[u].y * lda + x[u]];
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (pq[u].x < 0) continue;
          const float2 eaq = cmul(make_float2(R[u].z, -R[u].w), aq[u]);  // e^{i phi} a_q
          A[(long long)pq[u].x * lda + x[u]] =
              make_float2(R[u].x * ap[u].x - R[u].y * eaq.x, R[u].x * ap[u].y - R[u].y * eaq.y);
          A[(long long)pq[u].y * lda + x[u]] =
              make_float2(R[u].y * ap[u].x + R[u].x * eaq.x, R[u].y * ap[u].y + R[u].x * eaq.y);
        }
      }
      __syncthreads();
      // columns p, q: [A_.p, A_.q] J, and the same for Q (consecutive threads:
      // the pairs of one row); four rows per trip, loads first
      for (int e0 = threadIdx.x; e0 < npair * N; e0 += 4 * blockDim.x) {
        int2 pq[4];
        float4 R[4];
        float2* Ax[4];
        float2* Qx[4];
        float2 ap[4], aq[4], qp[4], qq[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int e = e0 + u * blockDim.x;
          const int xr = e / npair, i = e - xr * npair;
          pq[u] = (e < npair * N) ? pairs[i] : make_int2(-1, -1);
          Ax[u] = A + (long long)xr * lda;
          Qx[u] = Q + (long long)xr * lda;
          if (pq[u].x >= 0) {
            R[u] = rot[i];
            ap[u] = Ax[u][pq[u].x];
            aq[u] = Ax[u][pq[u].y];
            qp[u] = Qx[u][pq[u].x];
            qq[u] = Qx[u][pq[u].y];
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (pq[u].x < 0) continue;
          const float2 em = make_float2(R[u].z, R[u].w);  // e^{-i phi}
          const float2 eaq = cmul(em, aq[u]), eqq = cmul(em, qq[u]);
          const float c = R[u].x, sn = R[u].y;
          Ax[u][pq[u].x] = make_float2(c * ap[u].x - sn * eaq.x, c * ap[u].y - sn * eaq.y);
          Ax[u][pq[u].y] = make_float2(sn * ap[u].x + c * eaq.x, sn * ap[u].y + c * eaq.y);
          Qx[u][pq[u].x] = make_float2(c * qp[u].x - sn * eqq.x, c * qp[u].y - sn * eqq.y);
          Qx[u][pq[u].y] = make_float2(sn * qp[u].x + c * eqq.x, sn * qp[u].y + c * eqq.y);
        }
      }
      __syncthreads();
    }
  }
}

__global__ void __launch_bounds__(kThreads) wmmse_kernel(IterParams p, float bisect_tol, int bisect_max, int eig) {
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
      float2* Vk = sV + (long long)k * Nt * ldv;
      if (eig) {
        // A_k = Q diag(l) Q^H (Q in M), Y = Q^H B_k (in X), w_i = ||row i of Y||^2
        block_jacobi_eig(sA, sM, lda, Nt, reinterpret_cast<float4*>(sX), red, 12);
        float lam_i = 0.f;
        if (tid < Nt) lam_i = sA[(long long)tid * lda + tid].x;
        block_cgemm<4, 4, 1>(Nt, n, Nt, sM, lda, sB, ldv,
                             [&](int r, int c, float2 v) { sX[(long long)r * ldv + c] = v; });
        __syncthreads();
        float* lam = reinterpret_cast<float*>(sA);  // A's storage is free now
        float* wgt = lam + Nt;
        if (tid < Nt) {
          lam[tid] = lam_i;
          float wsum = 0.f;
          for (int c = 0; c < n; ++c) wsum += cabs2(sX[(long long)tid * ldv + c]);
          wgt[tid] = wsum;
        }
        __syncthreads();
        // the multiplier, by warp 0: lambda = 0 when A_k + 0 I is positive
        // definite and the power fits, else the same bisection as below
        if (tid < 32) {
          auto power_at = [&](float mu, float* pw) -> bool {
            float s = 0.f;
            bool pd = true;
            for (int i = tid; i < Nt; i += 32) {
              const float den = lam[i] + mu;
              pd = pd && (den > 0.f);
              s += wgt[i] / (den * den);
            }
            *pw = warp_sum(s);
            return __all_sync(0xffffffffu, pd);
          };
          float pw = 0.f, mu = 0.f;
          const bool pd0 = power_at(0.f, &pw);
          if (!(pd0 && pw <= Pc[k])) {
            float lo = 0.f, hi = (float)(sqrt(bnorm2) / sqrt((double)Pc[k]));
            for (int bi = 0; bi < bisect_max && (hi - lo) >= bisect_tol; ++bi) {
              const float mid = 0.5f * (lo + hi);
              const bool pd = power_at(mid, &pw);
              if (!pd || pw > Pc[k]) lo = mid;
              else hi = mid;
            }
            mu = hi;
            if (!power_at(hi, &pw) && tid == 0) s_fail = kNumeric;
          }
          if (tid == 0) s_piv = mu;
        }
        __syncthreads();
        if (s_fail != kOk) break;
        const float mu = s_piv;
        for (int e = tid; e < Nt * n; e += blockDim.x) {
          const int q = e / n, c = e - q * n;
          sX[(long long)q * ldv + c] = cscale(sX[(long long)q * ldv + c], 1.f / (lam[q] + mu));
        }
        __syncthreads();
        // V_k = Q diag(1 / (l + lambda)) Q^H B_k
        block_cgemm<4, 4, 0>(Nt, n, Nt, sM, lda, sX, ldv,
                             [&](int r, int c, float2 v) { Vk[(long long)r * ldv + c] = v; });
        __syncthreads();
        continue;
      }
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
