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
//   S7  Vtilde = Vhat - gamma G, ||Vtilde_k||_F^2 (FP64 accumulation), projection (15).
#include <math.h>
#include <stdio.h>

#include "amm_internal.cuh"

namespace amm {

// ------------------------------------------------------------------ GEMM
// Block-wide complex GEMM with a (TM x TN) register tile per thread; the
// rows of a tile are r = tr + i*ntr and its columns c = tc + j*ntc, so a
// warp reads consecutive columns of B.  OPA = 0: A(r,p) = A[r*lda + p];
// OPA = 1: A(r,p) = conj(A[p*lda + r]).  epi(r, c, value) for r < M, c < N.
template <int TM, int TN, int OPA, class Epi>
__device__ __forceinline__ void block_cgemm(int M, int N, int KK, const float2* __restrict__ A, int lda,
                                            const float2* __restrict__ B, int ldb, Epi epi) {
  const int ntr = (M + TM - 1) / TM, ntc = (N + TN - 1) / TN;
  const int ntiles = ntr * ntc;
  for (int tile = threadIdx.x; tile < ntiles; tile += blockDim.x) {
    const int tr = tile / ntc, tc = tile - tr * ntc;
    const float2* Ap[TM];
    const float2* Bp[TN];
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      int r = tr + i * ntr;
      r = (r < M) ? r : 0;  // out-of-range rows read row 0; their results are dropped
      Ap[i] = (OPA == 0) ? A + (long long)r * lda : A + r;
    }
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int c = tc + j * ntc;
      c = (c < N) ? c : 0;
      Bp[j] = B + c;
    }
    float2 acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = make_float2(0.f, 0.f);
#pragma unroll 2
    for (int p = 0; p < KK; ++p) {
      float2 a[TM], bb[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = (OPA == 0) ? Ap[i][p] : Ap[i][(long long)p * lda];
#pragma unroll
      for (int j = 0; j < TN; ++j) bb[j] = Bp[j][(long long)p * ldb];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j)
          acc[i][j] = (OPA == 0) ? cfma(a[i], bb[j], acc[i][j]) : cjfma(a[i], bb[j], acc[i][j]);
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int r = tr + i * ntr;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int c = tc + j * ntc;
        if (r < M && c < N) epi(r, c, acc[i][j]);
      }
    }
  }
}

// ------------------------------------------------------- bulk staging
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// Copy `rows` rows of `cols` complex elements from global (row stride
// gld) to shared memory (row stride sld).  Rows whose addresses and length
// are 16-byte multiples go through the TMA bulk-copy engine
// (cp.async.bulk) tracked by one mbarrier; anything else is copied by the
// threads.  Every wait is bounded by spin_budget; on timeout the status
// flag is set.  Contains __syncthreads().
__device__ void stage_rows(float2* dst, int sld, const float2* src, long long gld, int rows, int cols,
                           uint64_t* mbar, unsigned& phase, long long spin_budget, int* fail) {
  const bool bulk = ((reinterpret_cast<uintptr_t>(src) & 15) == 0) && ((gld & 1) == 0) &&
                    ((reinterpret_cast<uintptr_t>(dst) & 15) == 0) && ((sld & 1) == 0) && ((cols & 1) == 0) &&
                    (cols > 0) && ((long long)rows * cols * 8 < (1 << 20));
  if (!bulk) {
    for (long long e = threadIdx.x; e < (long long)rows * cols; e += blockDim.x) {
      const int r = (int)(e / cols), c = (int)(e - (long long)r * cols);
      dst[(long long)r * sld + c] = src[(long long)r * gld + c];
    }
    __syncthreads();
    return;
  }
  const unsigned bytes = (unsigned)cols * 8u;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)),
                 "r"(bytes * (unsigned)rows)
                 : "memory");
  }
  __syncwarp();
  if (threadIdx.x < 32) {
    for (int r = threadIdx.x; r < rows; r += 32) {
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              smem_u32(dst + (long long)r * sld)),
          "l"(src + (long long)r * gld), "r"(bytes), "r"(smem_u32(mbar))
          : "memory");
    }
  }
  // bounded wait for the phase to complete: spin on test_wait for at most
  // spin_budget SM clock cycles
  unsigned done = 0;
  const long long t0 = clock64();
  while (true) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(phase)
        : "memory");
    if (done || clock64() - t0 > spin_budget) break;
  }
  if (!done) atomicExch(fail, kTimeout);
  phase ^= 1u;
  __syncthreads();
}

// ------------------------------------------------------- small FP64 solves
// One thread per user.  Q: packed upper triangle (a <= b, row-major) of the
// interference-plus-noise covariance; zo(a, s): own-stream block of Z.
// Outputs U (NR x DD), UW = U W^{II} (NR x DD) and log det(I + M).
template <int NR, int DD>
__device__ bool small_solve(const float2* Qp, const float2* Zrow0, int ldz, int own0, float2* U, float2* UW,
                            double* logdet, bool want_u) {
  dcx L[NR][NR];
  double inv[NR];
  {
    int q = 0;
    dcx Q[NR][NR];
#pragma unroll
    for (int a = 0; a < NR; ++a)
#pragma unroll
      for (int b = a; b < NR; ++b) {
        Q[a][b] = dc(Qp[q++]);
        Q[b][a] = dconj(Q[a][b]);
      }
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      double dj = Q[j][j].x;
#pragma unroll
      for (int k = 0; k < j; ++k) dj -= L[j][k].x * L[j][k].x + L[j][k].y * L[j][k].y;
      if (!(dj > 0.0)) return false;
      const double rj = rsqrt(dj);
      inv[j] = rj;
      L[j][j] = dc(dj * rj, 0.0);
#pragma unroll
      for (int i = j + 1; i < NR; ++i) {
        dcx s = Q[i][j];
#pragma unroll
        for (int k = 0; k < j; ++k) s = dfmsj(L[i][k], L[j][k], s);
        L[i][j] = dscale(s, rj);
      }
    }
  }
  // X = L^{-1} Z_own
  dcx X[NR][DD];
#pragma unroll
  for (int c = 0; c < DD; ++c)
#pragma unroll
    for (int i = 0; i < NR; ++i) {
      dcx s = dc(Zrow0[(long long)i * ldz + own0 + c]);
#pragma unroll
      for (int k = 0; k < i; ++k) s = dfms(L[i][k], X[k][c], s);
      X[i][c] = dscale(s, inv[i]);
    }
  // I + M = I + X^H X (lower part) and its Cholesky factor R
  dcx R[DD][DD];
  double rinv[DD];
  double pivprod = 1.0;
  {
    dcx A[DD][DD];
#pragma unroll
    for (int a = 0; a < DD; ++a)
#pragma unroll
      for (int b = 0; b <= a; ++b) {
        dcx s = dc(a == b ? 1.0 : 0.0, 0.0);
#pragma unroll
        for (int i = 0; i < NR; ++i) s = djfma(X[i][a], X[i][b], s);
        A[a][b] = s;  // (X^H X)[a][b] = sum_i conj(X[i][a]) X[i][b]
      }
#pragma unroll
    for (int j = 0; j < DD; ++j) {
      double dj = A[j][j].x;
#pragma unroll
      for (int k = 0; k < j; ++k) dj -= R[j][k].x * R[j][k].x + R[j][k].y * R[j][k].y;
      if (!(dj > 0.0)) return false;
      pivprod *= dj;
      const double rj = rsqrt(dj);
      rinv[j] = rj;
      R[j][j] = dc(dj * rj, 0.0);
#pragma unroll
      for (int i = j + 1; i < DD; ++i) {
        dcx s = A[i][j];
#pragma unroll
        for (int k = 0; k < j; ++k) s = dfmsj(R[i][k], R[j][k], s);
        R[i][j] = dscale(s, rj);
      }
    }
  }
  *logdet = log(pivprod);
  if (!want_u) return true;
  // UW = L^{-H} X = Q^{-1} Z_own
  dcx Y[NR][DD];
#pragma unroll
  for (int c = 0; c < DD; ++c)
#pragma unroll
    for (int i = NR - 1; i >= 0; --i) {
      dcx s = X[i][c];
#pragma unroll
      for (int k = i + 1; k < NR; ++k) s = dfms(dconj(L[k][i]), Y[k][c], s);
      Y[i][c] = dscale(s, inv[i]);
    }
  // (I+M)^{-1} = R^{-H} R^{-1}: Rinv lower triangular
  dcx Ri[DD][DD];
#pragma unroll
  for (int j = 0; j < DD; ++j) {
    Ri[j][j] = dc(rinv[j], 0.0);
#pragma unroll
    for (int i = j + 1; i < DD; ++i) {
      dcx s = dc(0.0, 0.0);
#pragma unroll
      for (int k = j; k < i; ++k) s = dfms(R[i][k], Ri[k][j], s);
      Ri[i][j] = dscale(s, rinv[i]);
    }
  }
  dcx Mi[DD][DD];
#pragma unroll
  for (int a = 0; a < DD; ++a)
#pragma unroll
    for (int b = 0; b < DD; ++b) {
      dcx s = dc(0.0, 0.0);
      const int k0 = a > b ? a : b;
#pragma unroll
      for (int k = 0; k < DD; ++k)
        if (k >= k0) s = djfma(Ri[k][a], Ri[k][b], s);
      Mi[a][b] = s;
    }
#pragma unroll
  for (int i = 0; i < NR; ++i)
#pragma unroll
    for (int c = 0; c < DD; ++c) {
      dcx s = dc(0.0, 0.0);
#pragma unroll
      for (int b = 0; b < DD; ++b) s = dfma(Y[i][b], Mi[b][c], s);
      U[i * DD + c] = tof(s);
      UW[i * DD + c] = tof(Y[i][c]);
    }
  return true;
}

__device__ bool small_solve_dispatch(int Nr, int d, const float2* Qp, const float2* Zrow0, int ldz, int own0,
                                     float2* U, float2* UW, double* logdet, bool want_u) {
#define AMM_SS(a, b) \
  if (Nr == a && d == b) return small_solve<a, b>(Qp, Zrow0, ldz, own0, U, UW, logdet, want_u);
  AMM_SS(1, 1)
  AMM_SS(2, 1) AMM_SS(2, 2)
  AMM_SS(3, 1) AMM_SS(3, 2) AMM_SS(3, 3)
  AMM_SS(4, 1) AMM_SS(4, 2) AMM_SS(4, 3) AMM_SS(4, 4)
#undef AMM_SS
  return false;
}

// ------------------------------------------------------- Lanczos ||F_k||_2
// Largest eigenvalue of the Lanczos tridiagonal T (diagonal a, off-diagonal
// b) by multisection on the Sturm count, run by warp 0 (FP32).
__device__ float tridiag_max_eig(const float* a, const float* b, int n) {
  const int lane = threadIdx.x & 31;
  float lo = a[0], hi = a[0];
  for (int i = 0; i < n; ++i) {
    const float r = (i > 0 ? fabsf(b[i - 1]) : 0.f) + (i + 1 < n ? fabsf(b[i]) : 0.f);
    lo = fmaxf(lo, a[i]);
    hi = fmaxf(hi, a[i] + r);
  }
  const float scale = fmaxf(fabsf(hi), 1e-30f);
  for (int round = 0; round < 8; ++round) {
    const float x = lo + (hi - lo) * (float)(lane + 1) / 33.f;
    // number of eigenvalues below x (negative pivots of T - x I)
    int below = 0;
    float q = a[0] - x;
    if (fabsf(q) < 1e-30f * scale) q = -1e-30f * scale;
    below += q < 0.f;
    for (int i = 1; i < n; ++i) {
      q = (a[i] - x) - b[i - 1] * b[i - 1] / q;
      if (fabsf(q) < 1e-30f * scale) q = -1e-30f * scale;
      below += q < 0.f;
    }
    const unsigned mask = __ballot_sync(0xffffffffu, below < n);  // some eigenvalue >= x
    if (mask == 0u) {
      hi = lo + (hi - lo) / 33.f;
    } else {
      const int l = 31 - __clz(mask);
      const float nlo = lo + (hi - lo) * (float)(l + 1) / 33.f;
      const float nhi = (l == 31) ? hi : lo + (hi - lo) * (float)(l + 2) / 33.f;
      lo = nlo;
      hi = nhi;
    }
  }
  return 0.5f * (lo + hi);
}

struct Views {
  const float2* H;  // cell block j at H + j*m*ldh
  int ldh;
  float2* Z[2];
  int ldz;
  float2* V[2];     // cell block j at V + j*Nt*ldv
  int ldv;
  float2* QL;       // Krylov basis (Lm+1) x Nt
};

// Lanczos with full reorthogonalisation on F_k x = Htilde_k^H D Htilde_k x.
// Returns lambda_max of the tridiagonal (a lower bound on ||F_k||_2 that is
// exact when the Krylov space is invariant).  Contains __syncthreads().
__device__ float lanczos_norm(const InstDesc& D, const Layout& Ly, const float2* Hk, int ldh, const float2* sU,
                              const float2* sP, const float* alpha_u, float2* QL, float2* y, float2* z, float2* w,
                              float* ta, float* tb, float2* h, double* red, float* bcast) {
  const int Nt = D.Nt, m = Ly.m, Nr = D.Nr, d = D.d;
  const int tid = threadIdx.x;
  // group of g threads per output row, g a power of two <= 32
  int g = 1;
  while (g < 32 && 2 * g * m <= (int)blockDim.x) g <<= 1;
  int gN = 1;
  while (gN < 32 && 2 * gN * Nt <= (int)blockDim.x) gN <<= 1;
  // fixed start vector: unit-modulus entries with golden-ratio phases
  const float rn = rsqrtf((float)Nt);
  for (int p = tid; p < Nt; p += blockDim.x) {
    float s, c;
    sincosf(6.2831853f * 0.6180339887f * (float)(p + 1), &s, &c);
    QL[p] = make_float2(c * rn, s * rn);
  }
  __syncthreads();
  const int Lm = Ly.Lm;
  int Leff = Lm;
  float beta_prev = 0.f;
  for (int j = 0; j < Lm; ++j) {
    const float2* q = QL + (long long)j * Nt;
    // y = Htilde_k q
    for (int e = tid; e < m * g; e += blockDim.x) {
      const int i = e / g, l = e - i * g;
      float2 acc = make_float2(0.f, 0.f);
      for (int p = l; p < Nt; p += g) acc = cfma(Hk[(long long)i * ldh + p], q[p], acc);
      for (int o = g >> 1; o > 0; o >>= 1) {
        acc.x += __shfl_down_sync(0xffffffffu, acc.x, o, g);
        acc.y += __shfl_down_sync(0xffffffffu, acc.y, o, g);
      }
      if (l == 0) y[i] = acc;
    }
    __syncthreads();
    // z_r = 2 alpha_r P_r (U_r^H y_r)
    for (int i = tid; i < m; i += blockDim.x) {
      const int r = i / Nr, a = i - r * Nr;
      const float2* Ur = sU + r * Nr * d;
      const float2* Pr = sP + r * Nr * d;
      float2 acc = make_float2(0.f, 0.f);
      for (int s = 0; s < d; ++s) {
        float2 ts = make_float2(0.f, 0.f);
        for (int b = 0; b < Nr; ++b) ts = cjfma(Ur[b * d + s], y[r * Nr + b], ts);
        acc = cfma(Pr[a * d + s], ts, acc);
      }
      z[i] = cscale(acc, 2.f * alpha_u[r]);
    }
    __syncthreads();
    // w = Htilde_k^H z
    for (int e = tid; e < Nt * gN; e += blockDim.x) {
      const int p = e / gN, l = e - p * gN;
      float2 acc = make_float2(0.f, 0.f);
      for (int i = l; i < m; i += gN) acc = cjfma(Hk[(long long)i * ldh + p], z[i], acc);
      for (int o = gN >> 1; o > 0; o >>= 1) {
        acc.x += __shfl_down_sync(0xffffffffu, acc.x, o, gN);
        acc.y += __shfl_down_sync(0xffffffffu, acc.y, o, gN);
      }
      if (l == 0) w[p] = acc;
    }
    __syncthreads();
    double part = 0.0;
    for (int p = tid; p < Nt; p += blockDim.x) part += (double)(q[p].x * w[p].x + q[p].y * w[p].y);
    const float aj = (float)block_sum(part, red);
    const float2* qm = (j > 0) ? QL + (long long)(j - 1) * Nt : q;
    for (int p = tid; p < Nt; p += blockDim.x) {
      float2 v = w[p];
      v = csub(v, cscale(q[p], aj));
      if (j > 0) v = csub(v, cscale(qm[p], beta_prev));
      w[p] = v;
    }
    __syncthreads();
    // two passes of classical Gram-Schmidt against q_0..q_j
    for (int pass = 0; pass < 2; ++pass) {
      for (int i = tid >> 5; i <= j; i += blockDim.x >> 5) {
        const float2* qi = QL + (long long)i * Nt;
        float2 acc = make_float2(0.f, 0.f);
        for (int p = tid & 31; p < Nt; p += 32) acc = cjfma(qi[p], w[p], acc);
        acc = warp_sum(acc);
        if ((tid & 31) == 0) h[i] = acc;
      }
      __syncthreads();
      for (int p = tid; p < Nt; p += blockDim.x) {
        float2 v = w[p];
        for (int i = 0; i <= j; ++i) v = csub(v, cmul(h[i], QL[(long long)i * Nt + p]));
        w[p] = v;
      }
      __syncthreads();
    }
    double nn = 0.0;
    for (int p = tid; p < Nt; p += blockDim.x) nn += (double)cabs2(w[p]);
    const float bj = (float)sqrt(block_sum(nn, red));
    if (tid == 0) {
      ta[j] = aj;
      tb[j] = bj;
    }
    if (j + 1 >= Lm || !(bj > 1e-6f * fabsf(aj))) {
      Leff = j + 1;
      break;
    }
    const float ib = 1.f / bj;
    float2* qn = QL + (long long)(j + 1) * Nt;
    for (int p = tid; p < Nt; p += blockDim.x) qn[p] = cscale(w[p], ib);
    beta_prev = bj;
    __syncthreads();
  }
  __syncthreads();
  if (tid < 32) {
    const float lam = tridiag_max_eig(ta, tb, Leff);
    if (tid == 0) *bcast = lam;
  }
  __syncthreads();
  return *bcast;
}

// ------------------------------------------------------------------ kernel
__global__ void __launch_bounds__(kThreads) iterate_kernel(IterParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t mbar;
  __shared__ int s_fail;
  __shared__ int s_ctrl[8];
  __shared__ float s_bcast;

  const int b = blockIdx.x;
  const InstDesc D = p.desc[b];
  Scalars* scg = p.sc + b;
  const int tid = threadIdx.x;
  const int C = D.C, K = D.K, Nt = D.Nt, Nr = D.Nr, d = D.d;
  const Layout Ly = plan_layout(D, p.smem_budget, p.lanczos_steps);
  const int m = Ly.m, n = Ly.n, Cn = Ly.Cn, CK = Ly.CK, np = Ly.np;

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
  float* cellf = reinterpret_cast<float*>(smem + Ly.off_cell);  // [0,16): gamma, [16,32): scale
  float2* sU = reinterpret_cast<float2*>(smem + Ly.off_U);
  float2* sUW = reinterpret_cast<float2*>(smem + Ly.off_UW);
  float2* sQ = reinterpret_cast<float2*>(smem + Ly.off_Q);
  double* sRho = reinterpret_cast<double*>(smem + Ly.off_rho);
  float2* ly = reinterpret_cast<float2*>(smem + Ly.off_y);
  float2* lz = reinterpret_cast<float2*>(smem + Ly.off_z);
  float2* lw = reinterpret_cast<float2*>(smem + Ly.off_w);
  float* ta = reinterpret_cast<float*>(smem + Ly.off_tri);
  float* tb = ta + (Ly.Lm + 1);
  float2* lh = reinterpret_cast<float2*>(smem + Ly.off_h);

  const float* alpha_u = p.alpha + D.u_off;
  const float* Pc = p.P + D.c_off;
  float* gamma_c = p.gamma_c + D.c_off;
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
  const int ldh = vw.ldh, ldv = vw.ldv, ldz = vw.ldz;

  // Z(V^{t-2}) is needed from t = 3 on (omega > 0); rebuild it once per launch.
  if (p.mode != kEvalWsr && p.extrapolate && s_ctrl[0] >= 3) {
    for (int j = 0; j < C; ++j) {
      float2* Zo = vw.Z[zc ^ 1] + j * n;
      block_cgemm<4, 4, 0>(m, n, Nt, vw.H + (long long)j * m * ldh, ldh, vw.V[cur ^ 1] + (long long)j * Nt * ldv,
                           ldv, [&](int r, int c, float2 v) { Zo[(long long)r * ldz + c] = v; });
    }
    __syncthreads();
  }

  const int n_iters = (p.mode == kEvalWsr) ? 1 : p.n_iters;
  double rho = 0.0;
  for (int it = 0; it < n_iters; ++it) {
    const int t = s_ctrl[0];
    const float omega = (p.extrapolate && t >= 3) ? (float)(t - 2) / (float)(t + 1) : 0.f;
    float2* Zc = vw.Z[zc];
    float2* Zp = vw.Z[zc ^ 1];
    // ---- S2: Z = H V^{t-1}
    for (int j = 0; j < C; ++j) {
      float2* Zo = Zc + j * n;
      block_cgemm<4, 4, 0>(m, n, Nt, vw.H + (long long)j * m * ldh, ldh, vw.V[cur] + (long long)j * Nt * ldv, ldv,
                           [&](int r, int c, float2 v) { Zo[(long long)r * ldz + c] = v; });
    }
    __syncthreads();
    // ---- S3a: interference-plus-noise covariance Q_r (upper triangle), sigma^2 = 1
    for (int e = tid; e < CK * np; e += blockDim.x) {
      const int r = e / np;
      int q = e - r * np, a = 0;
      while (q >= Nr - a) { q -= Nr - a; ++a; }
      const int bb = a + q;
      const int own0 = (r / K) * n + (r % K) * d;
      const float2* za = Zc + (long long)(r * Nr + a) * ldz;
      const float2* zb = Zc + (long long)(r * Nr + bb) * ldz;
      float2 acc = make_float2(a == bb ? 1.f : 0.f, 0.f);
      for (int c = 0; c < Cn; ++c) {
        if (c >= own0 && c < own0 + d) continue;
        acc = cjfma(zb[c], za[c], acc);  // z_a conj(z_b)
      }
      sQ[e] = acc;
    }
    __syncthreads();
    // ---- S3b/S4: FP64 small solves, one thread per user
    const bool want_u = (p.mode != kEvalWsr);
    for (int r = tid; r < CK; r += blockDim.x) {
      const int own0 = (r / K) * n + (r % K) * d;
      double ld = 0.0;
      const bool ok = small_solve_dispatch(Nr, d, sQ + r * np, Zc + (long long)r * Nr * ldz, ldz, own0,
                                           sU + r * Nr * d, sUW + r * Nr * d, &ld, want_u);
      if (!ok || !isfinite(ld)) atomicExch(&s_fail, kNumeric);
      sRho[r] = ok ? ld : 0.0;
    }
    __syncthreads();
    double part = 0.0;
    for (int r = tid; r < CK; r += blockDim.x) part += (double)alpha_u[r] * sRho[r];
    rho = block_sum(part, red);
    if (s_fail != kOk) break;
    if (p.mode == kEvalWsr) {
      if (tid == 0) p.wsr_out[b] = rho / 0.69314718055994530942;
      break;
    }
    // ---- stage test of Algorithm 3 and the stopping test (thread 0)
    if (tid == 0) {
      const double rp = scg->rho_prev;
      const bool have_prev = !isnan(rp);
      const double rel = have_prev ? fabs(rho - rp) / fabs(rp) : INFINITY;
      int stop = 0;
      if (p.mode == kTolerance && s_ctrl[3] == 2 && rel <= (double)p.eps2) stop = 1;
      int stage = s_ctrl[1], si = s_ctrl[2];
      if (!stop) {
        if (stage == 1) {
          const bool go = (p.switch_iter >= 1) ? (t >= p.switch_iter) : (rel <= (double)p.eps1);
          if (go) { stage = 2; si = 0; }
        }
        si += 1;
        s_ctrl[1] = stage;
        s_ctrl[2] = si;
        const int spectral = (p.step_rule == 1) || (p.step_rule == 0 && si <= p.tc);
        s_ctrl[6] = spectral | ((p.step_rule == 0 && si == p.tc) ? 2 : 0);
      }
      s_ctrl[4] = stop;
    }
    __syncthreads();
    if (s_ctrl[4]) break;
    const int stage = s_ctrl[1];
    const float2* sP = (stage == 2) ? sUW : sU;  // U W: W = I (stage I) or E^{-1} (stage II)
    // ---- S6: Y = 2 alpha P (U^H Zhat - S), written over Z(V^{t-2})
    for (int e = tid; e < CK * Cn; e += blockDim.x) {
      const int r = e / Cn, c = e - r * Cn;
      const int own0 = (r / K) * n + (r % K) * d;
      const float2* Ur = sU + r * Nr * d;
      const float2* Pr = sP + r * Nr * d;
      float2 zh[kMaxNr];
#pragma unroll
      for (int a = 0; a < kMaxNr; ++a) {
        if (a < Nr) {
          const long long idx = (long long)(r * Nr + a) * ldz + c;
          float2 v = Zc[idx];
          if (omega != 0.f) v = csub(cscale(v, 1.f + omega), cscale(Zp[idx], omega));
          zh[a] = v;
        }
      }
      float2 ts[kMaxNr];
#pragma unroll
      for (int s = 0; s < kMaxNr; ++s) {
        if (s < d) {
          float2 acc = make_float2((c - own0 == s) ? -1.f : 0.f, 0.f);
#pragma unroll
          for (int a = 0; a < kMaxNr; ++a)
            if (a < Nr) acc = cjfma(Ur[a * d + s], zh[a], acc);
          ts[s] = acc;
        }
      }
      const float sc2 = 2.f * alpha_u[r];
#pragma unroll
      for (int a = 0; a < kMaxNr; ++a) {
        if (a < Nr) {
          float2 acc = make_float2(0.f, 0.f);
#pragma unroll
          for (int s = 0; s < kMaxNr; ++s)
            if (s < d) acc = cfma(Pr[a * d + s], ts[s], acc);
          Zp[(long long)(r * Nr + a) * ldz + c] = cscale(acc, sc2);
        }
      }
    }
    __syncthreads();
    // ---- S5: step size per cell, eq. (16)
    const int sflag = s_ctrl[6];
    for (int k = 0; k < C; ++k) {
      float gk;
      if (sflag & 1) {
        const float lam = lanczos_norm(D, Ly, vw.H + (long long)k * m * ldh, ldh, sU, sP, alpha_u, vw.QL, ly, lz,
                                       lw, ta, tb, lh, red, &s_bcast);
        gk = (lam > 0.f) ? 1.f / lam : 0.f;
        if ((sflag & 2) && tid == 0) gamma_c[k] = gk;
      } else {
        gk = (p.gamma_user > 0.f) ? p.gamma_user : gamma_c[k];
      }
      if (tid == 0) cellf[k] = gk;
    }
    __syncthreads();
    // ---- S7: G_j = Htilde_j^H Y_j; Vtilde = Vhat - gamma G over V^{t-2}; projection
    for (int j = 0; j < C; ++j) {
      const float gj = cellf[j];
      const float2* Vc = vw.V[cur] + (long long)j * Nt * ldv;
      float2* Vn = vw.V[cur ^ 1] + (long long)j * Nt * ldv;
      float nrm = 0.f;
      block_cgemm<4, 4, 1>(Nt, n, m, vw.H + (long long)j * m * ldh, ldh, Zp + j * n, ldz,
                           [&](int r, int c, float2 g) {
                             const long long idx = (long long)r * ldv + c;
                             float2 vh = Vc[idx];
                             if (omega != 0.f) vh = csub(cscale(vh, 1.f + omega), cscale(Vn[idx], omega));
                             const float2 vt = csub(vh, cscale(g, gj));
                             Vn[idx] = vt;
                             nrm += cabs2(vt);
                           });
      const double s = block_sum((double)nrm, red);
      if (tid == 0) cellf[16 + j] = (s > (double)Pc[j]) ? (float)sqrt((double)Pc[j] / s) : 1.f;
    }
    __syncthreads();
    for (int j = 0; j < C; ++j) {
      const float sj = cellf[16 + j];
      if (sj != 1.f) {
        float2* Vn = vw.V[cur ^ 1] + (long long)j * Nt * ldv;
        for (int e = tid; e < Nt * n; e += blockDim.x) {
          const int r = e / n, c = e - r * n;
          Vn[(long long)r * ldv + c] = cscale(Vn[(long long)r * ldv + c], sj);
        }
      }
    }
    __syncthreads();
    cur ^= 1;
    zc ^= 1;
    if (tid == 0) {
      scg->rho_prev = rho;
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
