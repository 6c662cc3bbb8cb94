// Device routines shared by the solver kernels: block-wide complex GEMM,
// TMA bulk staging, the compensated covariance, the per-user Hermitian
// solves (FP64, float-float or FP32) and the Lanczos estimate of
// ||F_k||_2.  Included by each kernel translation unit.
#pragma once

#include <math.h>

#include <type_traits>

#include "amm_ff.cuh"
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

// Register tile of the plain-path block GEMMs: 1 = 4 x 4, 2 = 2 x 2,
// 3 = 4 x 2, 4 = 4 x 3, 5 = 2 x 5.  0 picks, for the shape, the tile whose
// slowest thread does the least work: rounds of tiles over the block times
// the tile's multiply-adds plus its operand loads per K step (a 4 x 2 tile
// over M = 140, N = 20 takes two rounds on some threads, a 4 x 3 tile one).
__host__ __device__ inline int gemm_tile_pick(int M, int N, int nb) {
  const int tm[5] = {4, 2, 4, 4, 2}, tn[5] = {4, 2, 2, 3, 5};
  int best = 1;
  long long best_cost = -1;
  for (int k = 0; k < 5; ++k) {
    const long long tiles = (long long)((M + tm[k] - 1) / tm[k]) * ((N + tn[k] - 1) / tn[k]);
    const long long rounds = (tiles + nb - 1) / nb;
    const long long cost = rounds * (4 * tm[k] * tn[k] + 2 * (tm[k] + tn[k]));
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = k + 1;
    }
  }
  return best;
}
__device__ __forceinline__ int gemm_tile_for(int opt, int M, int N) {
  if (opt >= 1 && opt <= 5) return opt;
  return gemm_tile_pick(M, N, (int)blockDim.x);
}

template <int OPA, class Epi>
__device__ __forceinline__ void block_cgemm_tiled(int tile, int M, int N, int KK, const float2* __restrict__ A,
                                                  int lda, const float2* __restrict__ B, int ldb, Epi epi) {
  if (tile == 2)
    block_cgemm<2, 2, OPA>(M, N, KK, A, lda, B, ldb, epi);
  else if (tile == 3)
    block_cgemm<4, 2, OPA>(M, N, KK, A, lda, B, ldb, epi);
  else if (tile == 4)
    block_cgemm<4, 3, OPA>(M, N, KK, A, lda, B, ldb, epi);
  else if (tile == 5)
    block_cgemm<2, 5, OPA>(M, N, KK, A, lda, B, ldb, epi);
  else
    block_cgemm<4, 4, OPA>(M, N, KK, A, lda, B, ldb, epi);
}

// Block-wide complex GEMM for operands in global memory: 64 x 64 output
// tiles, each thread a 4 x 4 register tile (rows ty + 16 i, columns
// tx + 16 j, so that a warp reads consecutive shared-memory words), K in
// chunks of 16 staged through two shared-memory buffers (stage: at least
// kStageElems float2); the global loads of the next chunk are in flight
// while the current one is multiplied.  Same OPA and epilogue contract as
// block_cgemm; blockDim.x must be 256.  Contains __syncthreads().
constexpr int kStageBM = 64, kStageBN = 64, kStageKC = 16, kStageLdA = kStageKC + 1;
constexpr int kStageElems = 2 * (kStageBM * kStageLdA + kStageKC * kStageBN);

template <int OPA, class Epi>
__device__ void block_cgemm_staged(int M, int N, int KK, const float2* __restrict__ A, int lda,
                                   const float2* __restrict__ B, int ldb, Epi epi, float2* stage) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float2* As[2] = {stage, stage + kStageBM * kStageLdA + kStageKC * kStageBN};
  float2* Bs[2] = {As[0] + kStageBM * kStageLdA, As[1] + kStageBM * kStageLdA};
  const int mt = (M + kStageBM - 1) / kStageBM, nt = (N + kStageBN - 1) / kStageBN;
  const int nch = (KK + kStageKC - 1) / kStageKC;
  constexpr int kPer = (kStageBM * kStageKC) / 256;  // elements of each tile a thread stages per chunk
  for (int tile = 0; tile < mt * nt; ++tile) {
    const int r0 = (tile / nt) * kStageBM, c0 = (tile % nt) * kStageBN;
    float2 ra[kPer], rb[kPer];
    auto load = [&](int ch) {
      const int k0 = ch * kStageKC;
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        const int e = tid + 256 * u;
        float2 va = make_float2(0.f, 0.f), vb = make_float2(0.f, 0.f);
        if (OPA == 0) {  // A(r, k) = A[r lda + k]: a row's 16 k consecutive
          const int r = e / kStageKC, k = e % kStageKC;
          if (r0 + r < M && k0 + k < KK) va = A[(long long)(r0 + r) * lda + k0 + k];
        } else {         // A(r, k) = conj(A[k lda + r]): a k row's 64 r consecutive
          const int k = e / kStageBM, r = e % kStageBM;
          if (r0 + r < M && k0 + k < KK) {
            va = A[(long long)(k0 + k) * lda + r0 + r];
            va.y = -va.y;
          }
        }
        const int kb = e / kStageBN, cbn = e % kStageBN;
        if (k0 + kb < KK && c0 + cbn < N) vb = B[(long long)(k0 + kb) * ldb + c0 + cbn];
        ra[u] = va;
        rb[u] = vb;
      }
    };
    auto store = [&](int buf) {
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        const int e = tid + 256 * u;
        if (OPA == 0) {
          const int r = e / kStageKC, k = e % kStageKC;
          As[buf][r * kStageLdA + k] = ra[u];
        } else {
          const int k = e / kStageBM, r = e % kStageBM;
          As[buf][r * kStageLdA + k] = ra[u];
        }
        Bs[buf][(e / kStageBN) * kStageBN + e % kStageBN] = rb[u];
      }
    };
    float2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) acc[i][jj] = make_float2(0.f, 0.f);
    load(0);
    store(0);
    __syncthreads();
    for (int ch = 0; ch < nch; ++ch) {
      const int buf = ch & 1;
      if (ch + 1 < nch) load(ch + 1);  // in flight during the products below
#pragma unroll 4
      for (int k = 0; k < kStageKC; ++k) {
        float2 a[4], bb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[buf][(ty + 16 * i) * kStageLdA + k];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) bb[jj] = Bs[buf][k * kStageBN + tx + 16 * jj];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) acc[i][jj] = cfma(a[i], bb[jj], acc[i][jj]);
      }
      if (ch + 1 < nch) store(buf ^ 1);
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = r0 + ty + 16 * i;
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const int c = c0 + tx + 16 * jj;
        if (r < M && c < N) epi(r, c, acc[i][jj]);
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
static __device__ __noinline__ void stage_rows(float2* dst, int sld, const float2* src, long long gld, int rows, int cols,
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
  if (!done) {
    // report, then let the copies in flight land before anything else uses
    // (or releases) this shared memory: a second wait with a fixed budget
    atomicExch(fail, kTimeout);
    const long long t1 = clock64();
    while (!done && clock64() - t1 < kDrainBudget) {
      asm volatile(
          "{\n\t.reg .pred p;\n\t"
          "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t}"
          : "=r"(done)
          : "r"(smem_u32(mbar)), "r"(phase)
          : "memory");
    }
  }
  phase ^= 1u;
  __syncthreads();
}

// ------------------------------------------------------- small Hermitian solves
// Complex arithmetic in the solve precision T (double by default, float on
// request).
template <class T>
struct Cx {
  T x, y;
};
template <class T>
__device__ __forceinline__ Cx<T> mk(T x, T y) {
  Cx<T> r;
  r.x = x;
  r.y = y;
  return r;
}
template <class T>
__device__ __forceinline__ Cx<T> from2(float2 a) { return mk<T>((T)a.x, (T)a.y); }
template <class T>
__device__ __forceinline__ Cx<T> cj(Cx<T> a) { return mk<T>(a.x, -a.y); }
template <class T>
__device__ __forceinline__ Cx<T> scl(Cx<T> a, T s) { return mk<T>(a.x * s, a.y * s); }
// c - a*b
template <class T>
__device__ __forceinline__ Cx<T> fms(Cx<T> a, Cx<T> b, Cx<T> c) {
  return mk<T>(fma(-a.x, b.x, fma(a.y, b.y, c.x)), fma(-a.x, b.y, fma(-a.y, b.x, c.y)));
}
// c - a*conj(b)
template <class T>
__device__ __forceinline__ Cx<T> fmsj(Cx<T> a, Cx<T> b, Cx<T> c) {
  return mk<T>(fma(-a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(-a.y, b.x, c.y)));
}
// c + conj(a)*b
template <class T>
__device__ __forceinline__ Cx<T> jfma(Cx<T> a, Cx<T> b, Cx<T> c) {
  return mk<T>(fma(a.x, b.x, fma(a.y, b.y, c.x)), fma(a.x, b.y, fma(-a.y, b.x, c.y)));
}
// c + a*b
template <class T>
__device__ __forceinline__ Cx<T> fmac(Cx<T> a, Cx<T> b, Cx<T> c) {
  return mk<T>(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
template <class T>
__device__ __forceinline__ float2 to2(Cx<T> a) { return make_float2((float)a.x, (float)a.y); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double l1p(double x) { return log1p(x); }
__device__ __forceinline__ float l1p(float x) { return log1pf(x); }

template <class T>
__device__ __forceinline__ Cx<T> shfl4(Cx<T> v, int src) {
  return mk<T>(__shfl_sync(0xffffffffu, v.x, src, 4), __shfl_sync(0xffffffffu, v.y, src, 4));
}

// Per-user solve by a group of 4 consecutive lanes; lane c of the group
// owns column c of Z_own, X, U W and U (c < d), and every lane keeps the
// small Cholesky factors.  Qp: packed upper triangle (a <= b, row-major) of
// the interference-plus-noise covariance Q; Zrow0: the user's first row of Z
// (row stride ldz), own-stream columns own0.. .  With L = chol(Q),
// X = L^{-1} Z_own and M = X^H X (so that W = E^{-1} = I + M):
//   UW = L^{-H} X = Q^{-1} Z_own,  U = UW (I+M)^{-1},
//   logdet = log det(I + M) = sum_j log1p(pivot_j - 1), the pivots of I + M
//   computed from M itself (no rounding of 1 + small).
// Every lane of the warp must call this (it shuffles); `act` is false for
// lanes without a user.  Returns false on a non-positive pivot.
template <class T, int NR, int DD>
__device__ bool small_solve_grp(int c, bool act, const float2* Qp, const float2* Zrow0, int ldz, int own0,
                                float2* U, float2* UW, double* logdet, bool want_u, bool want_ld) {
  bool ok = act;
  Cx<T> L[NR][NR];
  T inv[NR];
  {
    Cx<T> Q[NR][NR];
    int q = 0;
#pragma unroll
    for (int a = 0; a < NR; ++a)
#pragma unroll
      for (int b = a; b < NR; ++b) {
        Q[a][b] = act ? from2<T>(Qp[q]) : mk<T>(a == b ? (T)1 : (T)0, (T)0);
        Q[b][a] = cj(Q[a][b]);
        ++q;
      }
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      T dj = Q[j][j].x;
#pragma unroll
      for (int k = 0; k < j; ++k) dj -= L[j][k].x * L[j][k].x + L[j][k].y * L[j][k].y;
      if (!(dj > (T)0)) {
        ok = false;
        dj = (T)1;
      }
      const T rj = rsq(dj);
      inv[j] = rj;
      L[j][j] = mk<T>(dj * rj, (T)0);
#pragma unroll
      for (int i = j + 1; i < NR; ++i) {
        Cx<T> s = Q[i][j];
#pragma unroll
        for (int k = 0; k < j; ++k) s = fmsj(L[i][k], L[j][k], s);
        L[i][j] = scl(s, rj);
      }
    }
  }
  // this lane's column of X = L^{-1} Z_own
  const bool mine = act && c < DD;
  Cx<T> x[NR];
#pragma unroll
  for (int i = 0; i < NR; ++i) {
    Cx<T> s = mine ? from2<T>(Zrow0[(long long)i * ldz + own0 + c]) : mk<T>((T)0, (T)0);
#pragma unroll
    for (int k = 0; k < i; ++k) s = fms(L[i][k], x[k], s);
    x[i] = scl(s, inv[i]);
  }
  // column c of M = X^H X: M[a][c] = sum_i conj(X[i][a]) x[i]
  Cx<T> mcol[DD];
#pragma unroll
  for (int a = 0; a < DD; ++a) {
    Cx<T> s = mk<T>((T)0, (T)0);
#pragma unroll
    for (int i = 0; i < NR; ++i) s = jfma(shfl4(x[i], a), x[i], s);
    mcol[a] = s;
  }
  // every lane gathers M and factors I + M = R R^H
  Cx<T> R[DD][DD];
  T rinv[DD];
  T mypiv = (T)0;
  {
    Cx<T> A[DD][DD];
#pragma unroll
    for (int b = 0; b < DD; ++b)
#pragma unroll
      for (int a = 0; a < DD; ++a) A[a][b] = shfl4(mcol[a], b);
#pragma unroll
    for (int j = 0; j < DD; ++j) {
      T dm1 = A[j][j].x;  // pivot - 1
#pragma unroll
      for (int k = 0; k < j; ++k) dm1 -= R[j][k].x * R[j][k].x + R[j][k].y * R[j][k].y;
      if (!(dm1 > (T)-1)) {
        ok = false;
        dm1 = (T)0;
      }
      if (j == c) mypiv = dm1;
      const T dj = (T)1 + dm1;
      const T rj = rsq(dj);
      rinv[j] = rj;
      R[j][j] = mk<T>(dj * rj, (T)0);
#pragma unroll
      for (int i = j + 1; i < DD; ++i) {
        Cx<T> s = A[i][j];
#pragma unroll
        for (int k = 0; k < j; ++k) s = fmsj(R[i][k], R[j][k], s);
        R[i][j] = scl(s, rj);
      }
    }
  }
  // log det(I + M): lane c contributes log1p of pivot c, summed over the group
  double ld = (want_ld && c < DD) ? (double)l1p(mypiv) : 0.0;
  ld += __shfl_xor_sync(0xffffffffu, ld, 1, 4);
  ld += __shfl_xor_sync(0xffffffffu, ld, 2, 4);
  if (c == 0) *logdet = ld;
  if (!want_u) return ok;
  // this lane's column of UW = L^{-H} x
  Cx<T> y[NR];
#pragma unroll
  for (int i = NR - 1; i >= 0; --i) {
    Cx<T> s = x[i];
#pragma unroll
    for (int k = i + 1; k < NR; ++k) s = fms(cj(L[k][i]), y[k], s);
    y[i] = scl(s, inv[i]);
  }
  // column c of (I+M)^{-1}: R g = e_c, then R^H m = g
  Cx<T> g[DD], mi[DD];
#pragma unroll
  for (int i = 0; i < DD; ++i) {
    Cx<T> s = mk<T>(i == c ? (T)1 : (T)0, (T)0);
#pragma unroll
    for (int k = 0; k < i; ++k) s = fms(R[i][k], g[k], s);
    g[i] = scl(s, rinv[i]);
  }
#pragma unroll
  for (int i = DD - 1; i >= 0; --i) {
    Cx<T> s = g[i];
#pragma unroll
    for (int k = i + 1; k < DD; ++k) s = fms(cj(R[k][i]), mi[k], s);
    mi[i] = scl(s, rinv[i]);
  }
  // U[:, c] = sum_b UW[:, b] (I+M)^{-1}[b][c]
#pragma unroll
  for (int i = 0; i < NR; ++i) {
    Cx<T> s = mk<T>((T)0, (T)0);
#pragma unroll
    for (int b = 0; b < DD; ++b) s = fmac(shfl4(y[i], b), mi[b], s);
    if (mine && ok) {
      U[i * DD + c] = to2(s);
      UW[i * DD + c] = to2(y[i]);
    }
  }
  return ok;
}

template <class T>
static __device__ __noinline__ bool small_solve_dispatch(int Nr, int d, int c, bool act, const float2* Qp,
                                                         const float2* Zrow0, int ldz, int own0, float2* U,
                                                         float2* UW, double* logdet, bool want_u, bool want_ld) {
#define AMM_SS(a, b) \
  if (Nr == a && d == b) \
    return small_solve_grp<T, a, b>(c, act, Qp, Zrow0, ldz, own0, U, UW, logdet, want_u, want_ld);
  AMM_SS(1, 1)
  AMM_SS(2, 1) AMM_SS(2, 2)
  AMM_SS(3, 1) AMM_SS(3, 2) AMM_SS(3, 3)
  AMM_SS(4, 1) AMM_SS(4, 2) AMM_SS(4, 3) AMM_SS(4, 4)
#undef AMM_SS
  return false;
}

// Arithmetic of the eight-lane per-user solve: FP64 (double) or
// float-float (ff, amm_ff.cuh) behind one interface, so both run the same
// sequence of operations.  flip(v, f) = f ? -v : v; positive(v): v > 0 and
// finite; Lg: the type the log-determinant terms are summed in.
template <class R>
struct PairArith;

template <>
struct PairArith<double> {
  typedef double R;
  typedef double Lg;
  static __device__ __forceinline__ R fma(R a, R b, R c) { return ::fma(a, b, c); }
  static __device__ __forceinline__ R mul(R a, R b) { return a * b; }
  static __device__ __forceinline__ R add(R a, R b) { return a + b; }
  static __device__ __forceinline__ R neg(R a) { return -a; }
  static __device__ __forceinline__ R flip(R v, bool f) {  // on the sign bit: no FP64 instruction
    return __longlong_as_double(__double_as_longlong(v) ^ (f ? (long long)0x8000000000000000ull : 0ll));
  }
  static __device__ __forceinline__ R shfl(R v, int src) { return __shfl_sync(0xffffffffu, v, src); }
  static __device__ __forceinline__ R shfl_xor(R v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
  static __device__ __forceinline__ bool positive(R v) {  // on the bits: no FP64 compare
    const long long b = __double_as_longlong(v);
    return b > 0ll && b < 0x7ff0000000000000ll;
  }
  static __device__ __forceinline__ R rsqrt(R v) { return ::rsqrt(v); }
  static __device__ __forceinline__ R from_f(float x) { return (double)x; }
  static __device__ __forceinline__ R from_f2(float hi, float lo) { return (double)hi + (double)lo; }
  static __device__ __forceinline__ float to_f(R v) { return (float)v; }
  static __device__ __forceinline__ R one() { return 1.0; }
  static __device__ __forceinline__ R zero() { return 0.0; }
  static __device__ __forceinline__ Lg log1p_(R v) { return ::log1p(v); }
  static __device__ __forceinline__ Lg lshfl_xor(Lg v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
};

template <>
struct PairArith<ff> {
  typedef ff R;
  typedef float Lg;
  static __device__ __forceinline__ R fma(R a, R b, R c) { return ff_fma(a, b, c); }
  static __device__ __forceinline__ R mul(R a, R b) { return ff_mul(a, b); }
  static __device__ __forceinline__ R add(R a, R b) { return ff_add(a, b); }
  static __device__ __forceinline__ R neg(R a) { return ff_neg(a); }
  static __device__ __forceinline__ R flip(R v, bool f) { return f ? ff_neg(v) : v; }
  static __device__ __forceinline__ R shfl(R v, int src) {
    return ff_make(__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src));
  }
  static __device__ __forceinline__ R shfl_xor(R v, int m) {
    return ff_make(__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m));
  }
  static __device__ __forceinline__ bool positive(R v) {
    const unsigned b = __float_as_uint(v.hi);
    return (b >> 31) == 0u && b != 0u && b < 0x7f800000u;
  }
  static __device__ __forceinline__ R rsqrt(R v) { return ff_rsqrt(v); }
  static __device__ __forceinline__ R from_f(float x) { return ff_from(x); }
  static __device__ __forceinline__ R from_f2(float hi, float lo) { return ff_make(hi, lo); }
  static __device__ __forceinline__ float to_f(R v) { return v.hi; }  // hi is hi + lo rounded to float
  static __device__ __forceinline__ R one() { return ff_from(1.f); }
  static __device__ __forceinline__ R zero() { return ff_from(0.f); }
  // log1p(hi + lo) = log1p(hi) + lo / (1 + hi) to first order; float accuracy
  static __device__ __forceinline__ Lg log1p_(R v) { return log1pf(v.hi) + v.lo / (1.f + v.hi); }
  static __device__ __forceinline__ Lg lshfl_xor(Lg v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
};

// Per-user solve by eight lanes: lane (c, p) of the group works on the
// real (p = 0) or imaginary (p = 1) part of every complex value it computes,
// and the partner lane (lane ^ 4) supplies the other part by one exchange.
// An FP64 warp instruction costs the same for any number of active lanes, so
// the work per lane is what counts:
//   * both Cholesky factors are formed row-parallel (lane c computes row c,
//     the pivot of step j comes from lane j, and each finished column is
//     broadcast so that every lane ends with the whole factor);
//   * X = L^{-1} Z_own and UW = L^{-H} X are solved column-parallel (lane c,
//     column c), and M = X^H X likewise;
//   * U = UW (I + M)^{-1} is solved row-parallel (lane c, row c of UW, by
//     v R^H = w then u R = v), so (I + M)^{-1} is never formed;
//   * pivot tests compare bit patterns instead of issuing FP64 compares.
// Same algebra as small_solve_grp; A = PairArith<double> or PairArith<ff>.
template <class A, int NR, int DD>
__device__ bool small_solve_pair(int c, int p, bool act, const float2* Qp, const float2* Qlo, const float2* Zrow0,
                                 int ldz, int own0, float2* U, float2* UW, double* logdet, bool want_u, bool want_ld) {
  typedef typename A::R R;
  typedef typename A::Lg Lg;
  typedef Cx<R> C;
  const int lane = threadIdx.x & 31, gb = lane & ~7;
  // s v with s = +1 on the imaginary lane and -1 on the real lane
  auto sg = [&](R v) { return A::flip(v, p == 0); };
  // own part of conj(v)
  auto ownj = [&](C v) { return p ? A::flip(v.y, true) : v.x; };
  auto own = [&](C v) { return p ? v.y : v.x; };
  auto oth = [&](C v) { return p ? v.x : v.y; };
  auto join = [&](R o) {
    const R t = A::shfl_xor(o, 4);
    return p ? mk<R>(t, o) : mk<R>(o, t);
  };
  // the whole complex value v of the lanes of column col
  auto from_col = [&](C v, int col) {
    const int src = gb + 4 * p + col;
    return mk<R>(A::shfl(v.x, src), A::shfl(v.y, src));
  };
  // products by parts (a, b whole): own(a b) = a.x own(b) + s a.y oth(b),
  // own(conj(a) b) = a.x own(b) - s a.y oth(b), own(a conj(b)) = -s a.x own(b) + a.y oth(b)
  bool ok = act;

  // Q = L L^H, row c of L by lane c; afterwards every lane holds all of L
  C L[NR][NR];
  R inv[NR];
  {
    R t0[NR];  // own part of Q[c][j] = conj(Q[j][c]), j <= c (high + low parts)
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      float2 v = make_float2(0.f, 0.f), vl = make_float2(0.f, 0.f);
      if (j <= c && c < NR) {
        const int q = j * NR - (j * (j - 1)) / 2 + (c - j);
        v = act ? Qp[q] : make_float2(j == c ? 1.f : 0.f, 0.f);
        if (act) vl = Qlo[q];
      }
      t0[j] = A::from_f2(p ? -v.y : v.x, p ? -vl.y : vl.x);
    }
    C lrow[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      R t = t0[j];
#pragma unroll
      for (int k = 0; k < j; ++k)  // t -= own(L[c][k] conj(L[j][k]))
        t = A::fma(A::neg(L[j][k].x), own(lrow[k]), A::fma(sg(L[j][k].y), oth(lrow[k]), t));
      R dj = A::shfl(t, gb + j);  // the pivot, from the real lane of row j
      if (!A::positive(dj)) {
        ok = false;
        dj = A::one();
      }
      const R rj = A::rsqrt(dj);
      inv[j] = rj;
      lrow[j] = join(A::mul(t, rj));
#pragma unroll
      for (int i = j + 1; i < NR; ++i) L[i][j] = from_col(lrow[j], i);
    }
  }
  // column c of X = L^{-1} Z_own
  const bool mine = act && c < DD;
  C x[NR];
#pragma unroll
  for (int i = 0; i < NR; ++i) {
    const float2 zv = mine ? Zrow0[(long long)i * ldz + own0 + c] : make_float2(0.f, 0.f);
    R t = A::from_f(p ? zv.y : zv.x);
#pragma unroll
    for (int k = 0; k < i; ++k)
      t = A::fma(A::neg(L[i][k].x), own(x[k]), A::fma(A::neg(sg(L[i][k].y)), oth(x[k]), t));
    x[i] = join(A::mul(t, inv[i]));
  }
  // column c of M = X^H X; row c of M is its conjugate (M Hermitian)
  C mcol[DD];
#pragma unroll
  for (int a = 0; a < DD; ++a) {
    R t = A::zero();
#pragma unroll
    for (int i = 0; i < NR; ++i) {
      const C xa = from_col(x[i], a);
      t = A::fma(xa.x, own(x[i]), A::fma(A::neg(sg(xa.y)), oth(x[i]), t));
    }
    mcol[a] = join(t);
  }
  // I + M = R R^H, row c of R by lane c (pivots kept minus one for log1p)
  C Rf[DD][DD];
  R rinv[DD];
  R mypiv = A::zero();
  {
    C rrow[DD];
#pragma unroll
    for (int j = 0; j < DD; ++j) {
      R t = ownj(mcol[j]);
#pragma unroll
      for (int k = 0; k < j; ++k) t = A::fma(A::neg(Rf[j][k].x), own(rrow[k]), A::fma(sg(Rf[j][k].y), oth(rrow[k]), t));
      R dm1 = A::shfl(t, gb + j);  // pivot - 1
      R dj = A::add(A::one(), dm1);
      if (!A::positive(dj)) {
        ok = false;
        dm1 = A::zero();
        dj = A::one();
      }
      if (j == c) mypiv = dm1;
      const R rj = A::rsqrt(dj);
      rinv[j] = rj;
      rrow[j] = join(A::mul(t, rj));
#pragma unroll
      for (int i = j + 1; i < DD; ++i) Rf[i][j] = from_col(rrow[j], i);
    }
  }
  // log det(I + M): lane c contributes log1p of pivot c, summed over the columns
  Lg ld = (want_ld && c < DD) ? A::log1p_(mypiv) : (Lg)0;
  ld += A::lshfl_xor(ld, 1);
  ld += A::lshfl_xor(ld, 2);
  if (c == 0 && p == 0) *logdet = (double)ld;
  if (!want_u) return ok;
  // column c of UW = L^{-H} x
  C y[NR];
#pragma unroll
  for (int i = NR - 1; i >= 0; --i) {
    R t = own(x[i]);
#pragma unroll
    for (int k = i + 1; k < NR; ++k) t = A::fma(A::neg(L[k][i].x), own(y[k]), A::fma(sg(L[k][i].y), oth(y[k]), t));
    y[i] = join(A::mul(t, inv[i]));
    if (mine && ok) reinterpret_cast<float*>(UW + i * DD + c)[p] = A::to_f(own(y[i]));
  }
  // row c of UW (own parts), gathered from the column lanes
  R w[DD];
#pragma unroll
  for (int b = 0; b < DD; ++b) w[b] = A::zero();
#pragma unroll
  for (int i = 0; i < NR; ++i)
#pragma unroll
    for (int b = 0; b < DD; ++b) {
      const R v = A::shfl(own(y[i]), gb + 4 * p + b);
      if (i == c) w[b] = v;
    }
  // row c of U = UW (R R^H)^{-1}: v R^H = w, then u R = v
  C v[DD], u[DD];
#pragma unroll
  for (int j = 0; j < DD; ++j) {
    R t = w[j];
#pragma unroll
    for (int k = 0; k < j; ++k)  // t -= own(v_k conj(R[j][k]))
      t = A::fma(sg(v[k].x), own(Rf[j][k]), A::fma(A::neg(v[k].y), oth(Rf[j][k]), t));
    v[j] = join(A::mul(t, rinv[j]));
  }
#pragma unroll
  for (int j = DD - 1; j >= 0; --j) {
    R t = own(v[j]);
#pragma unroll
    for (int k = j + 1; k < DD; ++k)  // t -= own(u_k R[k][j])
      t = A::fma(A::neg(u[k].x), own(Rf[k][j]), A::fma(A::neg(sg(u[k].y)), oth(Rf[k][j]), t));
    u[j] = join(A::mul(t, rinv[j]));
    if (act && ok && c < NR) reinterpret_cast<float*>(U + c * DD + j)[p] = A::to_f(own(u[j]));
  }
  return ok;
}

template <class A>
static __device__ __noinline__ bool small_solve_pair_dispatch(int Nr, int d, int c, int p, bool act,
                                                              const float2* Qp, const float2* Qlo,
                                                              const float2* Zrow0, int ldz, int own0, float2* U,
                                                              float2* UW, double* logdet, bool want_u,
                                                              bool want_ld) {
#define AMM_SP(a, b) \
  if (Nr == a && d == b) \
    return small_solve_pair<A, a, b>(c, p, act, Qp, Qlo, Zrow0, ldz, own0, U, UW, logdet, want_u, want_ld);
  AMM_SP(1, 1)
  AMM_SP(2, 1) AMM_SP(2, 2)
  AMM_SP(3, 1) AMM_SP(3, 2) AMM_SP(3, 3)
  AMM_SP(4, 1) AMM_SP(4, 2) AMM_SP(4, 3) AMM_SP(4, 4)
#undef AMM_SP
  return false;
}

// ------------------------------------------------------- Lanczos ||F_k||_2
// Number of eigenvalues of the symmetric tridiagonal T (diagonal a,
// off-diagonal b, order n) below x, by Sylvester's law of inertia: the
// number of negative pivots of T - x I, i.e. of sign changes in the
// sequence of leading principal minors p_i = det(T_{0..i} - x I), which obey
// the three-term recurrence p_i = (a_i - x) p_{i-1} - b_{i-1}^2 p_{i-2}.
// With T scaled by 1/scale (scale at least about the spectral radius) the
// entries are O(1), and every second step (p_i, p_{i-1}) is rescaled by an
// exact power of two, so the values stay in the FP32 range.  The serial
// chain is one FMA per step (no division); a zero minor counts as positive,
// which gives the same total as pushing a zero pivot to the negative side.
static __device__ __forceinline__ int sturm_below(const float* a, const float* b, int n, float x, float scale) {
  const float inv = 1.f / scale;
  float pm = 1.f, p = (a[0] - x) * inv;
  int below = (int)(__float_as_uint(p) >> 31);
  auto step = [&](float ai, float bi) {
    const float bs = bi * inv;
    const float pn = fmaf((ai - x) * inv, p, -(bs * bs) * pm);
    below += (int)((__float_as_uint(pn) ^ __float_as_uint(p)) >> 31);
    pm = p;
    p = pn;
  };
  auto renorm = [&]() {
    const unsigned e = (__float_as_uint(fmaxf(fabsf(p), fabsf(pm))) >> 23) & 0xffu;
    if (e >= 1u && e <= 253u) {
      const float f = __uint_as_float((254u - e) << 23);  // 2^(127 - e): exact
      p *= f;
      pm *= f;
    }
  };
  // four steps per trip with their entries loaded up front
  int i = 1;
  for (; i + 3 < n; i += 4) {
    const float a1 = a[i], a2 = a[i + 1], a3 = a[i + 2], a4 = a[i + 3];
    const float b1 = b[i - 1], b2 = b[i], b3 = b[i + 1], b4 = b[i + 2];
    step(a1, b1);
    step(a2, b2);
    renorm();
    step(a3, b3);
    step(a4, b4);
    renorm();
  }
  for (; i < n; ++i) {
    step(a[i], b[i - 1]);
    if ((i & 1) == 0) renorm();
  }
  return below;
}

// Gershgorin upper bound of the spectrum of T.
static __device__ __forceinline__ float tridiag_gershgorin(const float* a, const float* b, int n) {
  float hi = a[0];
#pragma unroll 4
  for (int i = 0; i < n; ++i) {
    const float r = (i > 0 ? fabsf(b[i - 1]) : 0.f) + (i + 1 < n ? fabsf(b[i]) : 0.f);
    hi = fmaxf(hi, a[i] + r);
  }
  return hi;
}

// Multisection on the Sturm count by warp 0, 32 points per round: narrows a
// bracket [lo, hi] that holds the largest eigenvalue of T (order n) down to
// FP32 resolution.  Returns the final bracket (x = lower end, y = upper end).
static __device__ __forceinline__ float2 tridiag_top_refine(const float* a, const float* b, int n, float lo, float hi) {
  const int lane = threadIdx.x & 31;
  if (hi < lo) hi = lo;
  const float scale = fmaxf(fabsf(hi), 1e-30f);
  for (int round = 0; round < 8 && hi - lo > 1.2e-7f * hi; ++round) {
    const float x = lo + (hi - lo) * (float)(lane + 1) / 33.f;
    const unsigned mask = __ballot_sync(0xffffffffu, sturm_below(a, b, n, x, scale) < n);  // some eigenvalue >= x
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
  return make_float2(lo, hi);
}

// Relative tolerance on the largest Ritz value between two checks, and the
// size of b_j, relative to the largest a_j, below which the Krylov space
// counts as invariant (what remains of w is then FP32 rounding).
constexpr float kLanczosTol = 1e-6f;
constexpr float kLanczosBreak = 1e-5f;

// Convergence check of the largest Ritz value, warp 0.  *lb holds a lower
// bound of the largest eigenvalue of the previous check's T, accurate to FP32
// resolution (0 before the first check).  By interlacing the largest Ritz
// value never decreases with the step, so *lb bounds the current T's from
// below too.  One Sturm round tests x_l = lb (1 + tol 2^l), l = 0..31: when
// no eigenvalue reaches x_0 the value moved by less than tol since the last
// check and the call returns true; otherwise the bracket between the
// highest x_l reached and the next one is refined and *lb rises to it.
static __device__ __forceinline__ bool tridiag_top_settled(const float* a, const float* b, int n, float* lb) {
  const int lane = threadIdx.x & 31;
  const float base = *lb;
  const float gh = tridiag_gershgorin(a, b, n);
  if (!(base > 0.f)) {
    float amax = a[0];
    for (int i = 1; i < n; ++i) amax = fmaxf(amax, a[i]);
    const float2 br = tridiag_top_refine(a, b, n, amax, gh);
    if (lane == 0) *lb = br.x;
    return false;
  }
  const float scale = fmaxf(fabsf(gh), 1e-30f);
  const float x = base * (1.f + kLanczosTol * ldexpf(1.f, lane));
  const unsigned mask = __ballot_sync(0xffffffffu, sturm_below(a, b, n, x, scale) < n);
  if ((mask & 1u) == 0u) return true;
  const int l = 31 - __clz(mask);
  const float lo = base * (1.f + kLanczosTol * ldexpf(1.f, l));
  const float hi = (l == 31) ? gh : base * (1.f + kLanczosTol * ldexpf(1.f, l + 1));
  const float2 br = tridiag_top_refine(a, b, n, lo, hi);
  __syncwarp();
  if (lane == 0) *lb = br.x;
  return false;
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

// Lanczos on F_k x = Htilde_k^H D Htilde_k x, D = blkdiag(2 alpha U W U^H),
// by the plain three-term recurrence
//   w = F_k q_j - a_j q_j - b_{j-1} q_{j-1},  a_j = q_j^H F_k q_j,  b_j = ||w||,
// without reorthogonalisation.  In floating point the basis loses
// orthogonality as Ritz values converge, but every Ritz value stays within
// the spectrum up to rounding (Paige's analysis of the finite-precision
// recurrence), so the largest one converges to ||F_k||_2 from below; the
// lost orthogonality only adds copies of converged values.  From step 12
// on, every third step tests whether the largest Ritz value still moves by
// more than kLanczosTol (tridiag_top_settled, by warp 0); the iteration ends
// there, at an invariant Krylov space (b_j below kLanczosBreak times the
// largest a_j) or at Ly.Lm steps.  q_{j+1} stays unnormalised in the slot
// of q_{j-1} and its scale 1/b_j is applied where it is read; QL holds the
// two slots (2 Nt).  FP32 reductions only.
__device__ __forceinline__ bool lanczos_check_due(int steps) { return steps >= 12 && (steps - 12) % 3 == 0; }

// D_r = 2 alpha_r P_r U_r^H (Nr x Nr per user) into sD, the fixed start
// vector (unit-modulus entries with golden-ratio phases) into slot 0 and
// q_{-1} = 0 into slot 1.  No barrier.
__device__ __forceinline__ void lanczos_setup(const InstDesc& D, const Layout& Ly, const float2* sU, const float2* sP,
                                              const float* alpha_u, float2* QL, float2* sD) {
  const int Nt = D.Nt, Nr = D.Nr, d = D.d;
  for (int e = threadIdx.x; e < Ly.CK * Nr * Nr; e += blockDim.x) {
    const int r = e / (Nr * Nr), ab = e - r * Nr * Nr, a = ab / Nr, b = ab - a * Nr;
    float2 acc = make_float2(0.f, 0.f);
    for (int s = 0; s < d; ++s) acc = cfma(sP[(r * Nr + a) * d + s], make_float2(sU[(r * Nr + b) * d + s].x,
                                                                              -sU[(r * Nr + b) * d + s].y), acc);
    sD[e] = cscale(acc, 2.f * alpha_u[r]);
  }
  const float rn = rsqrtf((float)Nt);
  for (int p = threadIdx.x; p < Nt; p += blockDim.x) {
    float s, c;
    sincosf(6.2831853f * 0.6180339887f * (float)(p + 1), &s, &c);
    QL[p] = make_float2(c * rn, s * rn);
    QL[Nt + p] = make_float2(0.f, 0.f);
  }
}

// The estimate of ||F_k||_2 once the steps have ended (warp 0 computes,
// every thread returns it): the settled lower bound, or the largest
// eigenvalue of T refined to FP32 resolution.  Contains __syncthreads().
__device__ __forceinline__ float lanczos_finish(const float* ta, const float* tb, int Leff, bool settled,
                                                const float* s_lb, float* bcast) {
  __syncthreads();
  if (threadIdx.x < 32) {
    float lam;
    if (settled) {
      lam = *s_lb * (1.f + 0.5f * kLanczosTol);
    } else {
      float lo = fmaxf(*s_lb, ta[0]);
      for (int i = 1; i < Leff; ++i) lo = fmaxf(lo, ta[i]);
      const float2 br = tridiag_top_refine(ta, tb, Leff, lo, tridiag_gershgorin(ta, tb, Leff));
      lam = 0.5f * (br.x + br.y);
    }
    if (threadIdx.x == 0) *bcast = lam;
  }
  __syncthreads();
  return *bcast;
}

// General form (any shape, hget(i, q) from shared or global memory): three
// barriers per step.  a_j = (Htilde q_j)^H D (Htilde q_j) is summed while
// z = D y is formed; w is formed, updated and its norm taken by the thread
// that owns its entry.  Contains __syncthreads().
template <class HGet>
__device__ float lanczos_norm(const InstDesc& D, const Layout& Ly, HGet hget, const float2* sU, const float2* sP,
                              const float* alpha_u, float2* QL, float2* y, float2* z, float2* sD, float* ta,
                              float* tb, double* red, float* bcast, bool h_global = false) {
  const int Nt = D.Nt, m = Ly.m, Nr = D.Nr;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  float* redf = reinterpret_cast<float*>(red);
  float* s_apart = redf;        // [nw] partial sums of a_j
  float* s_bpart = redf + 8;    // [nw] partial sums of b_j^2
  float* s_lb = redf + 32;      // lower bound of the largest Ritz value (warp 0)
  float* s_done = redf + 33;    // settled flag, read by every thread after a barrier
  // group of g threads per output row, g a power of two <= 32; a channel in
  // global memory is read a row per warp (coalesced) instead
  int g = 1;
  while (g < 32 && 2 * g * m <= (int)blockDim.x) g <<= 1;
  if (h_global && Nt >= 32) g = 32;
  int gN = 1;
  while (gN < 32 && 2 * gN * Nt <= (int)blockDim.x) gN <<= 1;
  float2* slot[2] = {QL, QL + Nt};
  lanczos_setup(D, Ly, sU, sP, alpha_u, QL, sD);
  if (tid == 0) {
    *s_lb = 0.f;
    *s_done = 0.f;
  }
  __syncthreads();
  const int Lm = Ly.Lm;
  int Leff = Lm;
  bool settled = false;
  float amax = 0.f;                // largest a_j so far (a lower bound of lambda_max)
  float sc_cur = 1.f, sc_prev = 0.f;  // q_j = sc_cur * slot[cur], q_{j-1} = sc_prev * slot[cur ^ 1]
  float bprev = 0.f;
  int cur = 0;
  for (int j = 0; j < Lm; ++j) {
    const float2* qj = slot[cur];
    // y = Htilde_k q_j
    for (int e0 = 0; e0 < m * g; e0 += blockDim.x) {  // warp-uniform trip count for the shuffles
      const int e = e0 + tid;
      const bool act = e < m * g;
      const int i = act ? e / g : 0, l = e % g;
      float2 acc = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
      if (act) {  // two independent chains
        int p = l;
        for (; p + g < Nt; p += 2 * g) {
          acc = cfma(hget(i, p), qj[p], acc);
          acc1 = cfma(hget(i, p + g), qj[p + g], acc1);
        }
        if (p < Nt) acc = cfma(hget(i, p), qj[p], acc);
        acc = cadd(acc, acc1);
      }
      for (int o = g >> 1; o > 0; o >>= 1) {
        acc.x += __shfl_down_sync(0xffffffffu, acc.x, o, g);
        acc.y += __shfl_down_sync(0xffffffffu, acc.y, o, g);
      }
      if (act && l == 0) y[i] = cscale(acc, sc_cur);
    }
    __syncthreads();
    if (*s_done != 0.f) {  // set by the previous step's check
      settled = true;
      break;
    }
    // z_r = D_r y_r, and a_j = sum_i Re(conj(y_i) z_i)
    float apart = 0.f;
    for (int i = tid; i < m; i += blockDim.x) {
      const int r = i / Nr, a = i - r * Nr;
      const float2* Dr = sD + (r * Nr + a) * Nr;
      float2 zi = make_float2(0.f, 0.f);
      for (int b = 0; b < Nr; ++b) zi = cfma(Dr[b], y[r * Nr + b], zi);
      z[i] = zi;
      const float2 yi = y[i];
      apart = fmaf(yi.x, zi.x, fmaf(yi.y, zi.y, apart));
    }
    apart = warp_sum(apart);
    if (lane == 0) s_apart[warp] = apart;
    __syncthreads();
    float aj = 0.f;
    for (int q2 = 0; q2 < nw; ++q2) aj += s_apart[q2];  // same order in every thread
    // w = Htilde_k^H z - a_j q_j - b_{j-1} q_{j-1}, into the slot of q_{j-1}
    float2* qn = slot[cur ^ 1];
    float bpart = 0.f;
    for (int e0 = 0; e0 < Nt * gN; e0 += blockDim.x) {
      const int e = e0 + tid;
      const bool act = e < Nt * gN;
      const int p = act ? e / gN : 0, l = e % gN;
      float2 acc = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
      if (act) {  // two independent chains
        int i = l;
        for (; i + gN < m; i += 2 * gN) {
          acc = cjfma(hget(i, p), z[i], acc);
          acc1 = cjfma(hget(i + gN, p), z[i + gN], acc1);
        }
        if (i < m) acc = cjfma(hget(i, p), z[i], acc);
        acc = cadd(acc, acc1);
      }
      for (int o = gN >> 1; o > 0; o >>= 1) {
        acc.x += __shfl_down_sync(0xffffffffu, acc.x, o, gN);
        acc.y += __shfl_down_sync(0xffffffffu, acc.y, o, gN);
      }
      if (act && l == 0) {
        const float2 v = csub(csub(acc, cscale(qj[p], aj * sc_cur)), cscale(qn[p], bprev * sc_prev));
        qn[p] = v;
        bpart += cabs2(v);
      }
    }
    bpart = warp_sum(bpart);
    if (lane == 0) s_bpart[warp] = bpart;
    __syncthreads();
    float ss = 0.f;
    for (int q2 = 0; q2 < nw; ++q2) ss += s_bpart[q2];
    const float bj = sqrtf(ss);
    if (tid == 0) {
      ta[j] = aj;
      tb[j] = bj;
    }
    amax = fmaxf(amax, aj);
    // an invariant Krylov space: what is left of w is rounding noise
    if (j + 1 >= Lm || !(bj > kLanczosBreak * amax)) {
      Leff = j + 1;
      break;
    }
    sc_prev = sc_cur;
    sc_cur = 1.f / bj;
    bprev = bj;
    cur ^= 1;
    // convergence check on T_{j+1}; the verdict is read after the next barrier
    if (warp == 0 && lanczos_check_due(j + 1)) {
      __syncwarp();  // ta[j], tb[j] from lane 0
      const bool done = tridiag_top_settled(ta, tb, j + 1, s_lb);
      if (lane == 0 && done) *s_done = 1.f;
    }
  }
  return lanczos_finish(ta, tb, Leff, settled, s_lb, bcast);
}

// Sum over the 32 lanes of eight complex values per lane, scattered: lane l
// returns the total of value l >> 2 (the four lanes of a group agree).  18
// shuffles instead of 80 for eight separate warp sums; a fixed order.
__device__ __forceinline__ float2 warp_reduce_scatter8(const float2 (&v)[8]) {
  const int lane = threadIdx.x & 31;
  float2 u[4], w2[2];
  const bool b16 = lane & 16, b8 = lane & 8, b4 = lane & 4;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 snd = b16 ? v[k] : v[k + 4], keep = b16 ? v[k + 4] : v[k];
    u[k] = make_float2(keep.x + __shfl_xor_sync(0xffffffffu, snd.x, 16),
                       keep.y + __shfl_xor_sync(0xffffffffu, snd.y, 16));
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float2 snd = b8 ? u[k] : u[k + 2], keep = b8 ? u[k + 2] : u[k];
    w2[k] = make_float2(keep.x + __shfl_xor_sync(0xffffffffu, snd.x, 8),
                        keep.y + __shfl_xor_sync(0xffffffffu, snd.y, 8));
  }
  const float2 snd = b4 ? w2[0] : w2[1], keep = b4 ? w2[1] : w2[0];
  float2 x = make_float2(keep.x + __shfl_xor_sync(0xffffffffu, snd.x, 4),
                         keep.y + __shfl_xor_sync(0xffffffffu, snd.y, 4));
  x.x += __shfl_xor_sync(0xffffffffu, x.x, 2);
  x.y += __shfl_xor_sync(0xffffffffu, x.y, 2);
  x.x += __shfl_xor_sync(0xffffffffu, x.x, 1);
  x.y += __shfl_xor_sync(0xffffffffu, x.y, 1);
  return x;
}

// Users per warp of the row-blocked form below.
__host__ __device__ inline int lanczos_users_per_warp(const Layout& Ly, int nw) { return (Ly.CK + nw - 1) / nw; }
// Whether the row-blocked form applies: 256 threads, Nt <= 64, at most 64
// rows, and each warp's users spanning at most eight rows.
__host__ __device__ inline bool lanczos_rows_ok(const InstDesc& D, const Layout& Ly, int threads) {
  const int nw = threads / 32;
  return threads == 256 && D.Nt <= 64 && Ly.m <= 64 && D.Nr * lanczos_users_per_warp(Ly, nw) <= 8;
}

// Row-blocked form when lanczos_rows_ok holds: Htilde (row stride ldh, in
// global or shared memory) is read once into registers, and a step costs
// two barriers and no further reads of it.  Warp w owns the rows of its
// users, its lanes the columns l and l + 32 of those rows.  One
// reduce-scatter leaves y_i = (Htilde q_j)_i with the four lanes of row i,
// so z = D y and the warp's part of a_j follow by shuffles within the warp;
// the warp's part of Htilde^H z (its rows only) goes to wpart (nw x 64),
// and after the barrier the threads of column p sum the nw parts in warp
// order, form w, its entry of q_{j+1} and their part of b_j^2.  zbuf: m
// entries.  Same recurrence, tests and scratch as lanczos_norm otherwise.
// Not inlined: the registers holding Htilde are its own, not the caller's.
// Contains __syncthreads().
static __device__ __noinline__ float lanczos_norm_rows(const InstDesc& D, const Layout& Ly, const float2* Hg, int ldh,
                                                       const float2* sU, const float2* sP, const float* alpha_u,
                                                       float2* QL, float2* zbuf, float2* wpart, float2* sD,
                                                       float* ta, float* tb, double* red, float* bcast) {
  constexpr int nw = 8;  // lanczos_rows_ok: 256 threads
  const int Nt = D.Nt, m = Ly.m, Nr = D.Nr;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float* redf = reinterpret_cast<float*>(red);
  float* s_apart = redf;        // [nw] partial sums of a_j
  float* s_bpart = redf + 8;    // [2] partial sums of b_j^2 (the column warps)
  float* s_lb = redf + 32;
  float* s_done = redf + 33;
  const int upw = lanczos_users_per_warp(Ly, nw);
  const int row0 = warp * upw * Nr;          // first row of this warp's users
  const int nrow = min(upw * Nr, m - row0);  // rows of this warp (may be <= 0)
  const int k4 = lane >> 2;                  // the row a lane holds after the reduce-scatter
  const bool lead = (lane & 3) == 0;
  const int ncw = (Nt + 31) >> 5;            // warps that combine the columns (1 or 2)
  float2* slot[2] = {QL, QL + Nt};
  // this warp's rows of Htilde, columns lane and lane + 32
  float2 h0[8], h1[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float2* hr = Hg + (long long)(row0 + k) * ldh;
    h0[k] = (k < nrow && lane < Nt) ? hr[lane] : make_float2(0.f, 0.f);
    h1[k] = (k < nrow && lane + 32 < Nt) ? hr[lane + 32] : make_float2(0.f, 0.f);
  }
  lanczos_setup(D, Ly, sU, sP, alpha_u, QL, sD);
  if (tid == 0) {
    *s_lb = 0.f;
    *s_done = 0.f;
  }
  __syncthreads();
  // the lane's row of its user's D_r (row k4 after the reduce-scatter), and
  // the lanes that hold the user's y entries; zero beyond Nr
  const int u = k4 / Nr, a = k4 - u * Nr, r = warp * upw + u;
  const bool valid = k4 < nrow && r < Ly.CK;
  float2 dr[kMaxNr];
  int ysrc[kMaxNr];
#pragma unroll
  for (int b = 0; b < kMaxNr; ++b) {
    dr[b] = (valid && b < Nr) ? sD[(r * Nr + a) * Nr + b] : make_float2(0.f, 0.f);
    ysrc[b] = min(4 * (u * Nr + b) + (lane & 3), 31);
  }
  const int Lm = Ly.Lm;
  int Leff = Lm;
  bool settled = false;
  float amax = 0.f;
  float sc_cur = 1.f, sc_prev = 0.f;
  float bprev = 0.f;
  int cur = 0;
  for (int j = 0; j < Lm; ++j) {
    const float2* qj = slot[cur];
    // ---- y = Htilde q_j over this warp's rows, z = D y, a_j's part and
    //      this warp's part of Htilde^H z
    {
      const float2 q0 = (lane < Nt) ? cscale(qj[lane], sc_cur) : make_float2(0.f, 0.f);
      const float2 q1 = (lane + 32 < Nt) ? cscale(qj[lane + 32], sc_cur) : make_float2(0.f, 0.f);
      float2 acc[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[k] = cfma(h1[k], q1, cmul(h0[k], q0));
      const float2 yk = warp_reduce_scatter8(acc);  // y of local row k4 (zero beyond nrow)
      // z_i = sum_b D_r[a][b] y_{r Nr + b}: the rows of user u sit in lanes 4 (u Nr + b) + (lane & 3)
      float2 yb[kMaxNr];
#pragma unroll
      for (int b = 0; b < kMaxNr; ++b)
        yb[b] = make_float2(__shfl_sync(0xffffffffu, yk.x, ysrc[b]), __shfl_sync(0xffffffffu, yk.y, ysrc[b]));
      float2 zk = make_float2(0.f, 0.f);
#pragma unroll
      for (int b = 0; b < kMaxNr; ++b) zk = cfma(dr[b], yb[b], zk);  // zero beyond Nr and for invalid rows
      if (valid && lead) zbuf[row0 + k4] = zk;
      __syncwarp();
      float2 w0 = make_float2(0.f, 0.f), w1 = make_float2(0.f, 0.f);
      if (nrow > 0) {  // rows past nrow hold zero channel entries: clamp their index, keep the sum
        float2 zr[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) zr[k] = zbuf[row0 + min(k, nrow - 1)];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          w0 = cjfma(h0[k], zr[k], w0);
          w1 = cjfma(h1[k], zr[k], w1);
        }
      }
      wpart[warp * 64 + lane] = w0;
      wpart[warp * 64 + 32 + lane] = w1;
      float apart = lead ? fmaf(yk.x, zk.x, yk.y * zk.y) : 0.f;
      apart = warp_sum(apart);
      if (lane == 0) s_apart[warp] = apart;
    }
    __syncthreads();
    if (*s_done != 0.f) {  // set by the previous step's check
      settled = true;
      break;
    }
    float aj = 0.f;
#pragma unroll
    for (int q2 = 0; q2 < nw; ++q2) aj += s_apart[q2];  // same order in every thread
    // ---- w = Htilde^H z - a_j q_j - b_{j-1} q_{j-1}: thread p sums the parts in warp order
    float2* qn = slot[cur ^ 1];
    if (warp < ncw) {
      float bpart = 0.f;
      if (tid < Nt) {
        float2 gp[nw];
#pragma unroll
        for (int q2 = 0; q2 < nw; ++q2) gp[q2] = wpart[q2 * 64 + tid];
        float2 g = gp[0];
#pragma unroll
        for (int q2 = 1; q2 < nw; ++q2) g = cadd(g, gp[q2]);
        const float2 v = csub(csub(g, cscale(qj[tid], aj * sc_cur)), cscale(qn[tid], bprev * sc_prev));
        qn[tid] = v;
        bpart = cabs2(v);
      }
      bpart = warp_sum(bpart);
      if (lane == 0) s_bpart[warp] = bpart;
    }
    __syncthreads();
    float ss = s_bpart[0];
    if (ncw > 1) ss += s_bpart[1];
    const float bj = sqrtf(ss);
    if (tid == 0) {
      ta[j] = aj;
      tb[j] = bj;
    }
    amax = fmaxf(amax, aj);
    if (j + 1 >= Lm || !(bj > kLanczosBreak * amax)) {
      Leff = j + 1;
      break;
    }
    sc_prev = sc_cur;
    sc_cur = 1.f / bj;
    bprev = bj;
    cur ^= 1;
    if (warp == 0 && lanczos_check_due(j + 1)) {
      __syncwarp();
      const bool done = tridiag_top_settled(ta, tb, j + 1, s_lb);
      if (lane == 0 && done) *s_done = 1.f;
    }
  }
  return lanczos_finish(ta, tb, Leff, settled, s_lb, bcast);
}

// ------------------------------------------------------- per-user phases
// S3a: upper triangle of Q_r = sigma^2 I + sum over streams other than the
// user's own of z z^H (sigma^2 = 1 after normalisation).  zget(row, col).
// Entries of z z^H summed over many streams can be far larger than the
// noise term (about 1e6 against 1 for a cell-centre user of the seven-cell
// layout), where FP32 rounding of the sum would blur the noise floor that
// eq. (9) resolves; so each entry is a compensated dot product (the
// products split exactly by FMA, the sums by two_sum, the rounding errors
// accumulated separately: about twice FP32 precision), stored as a high
// part (sQ, read by the FP32 solves) and a low part (sQ + CK np, read by
// the FP64 and float-float solves).
// One entry sum_c z_a(c) conj(z_b(c)) over columns [c0, c1) except
// [skip0, skip1), as a compensated dot product (the products split exactly by
// FMA, the sums by two_sum, the rounding errors accumulated apart): about
// twice FP32 precision.  Four interleaved chains per part keep the FP32 pipe
// busy; zget(row, col).  Returns (re, im) in float-float.
template <class ZGet>
__device__ __forceinline__ void cov_entry(ZGet zget, int ra, int rb, int c0, int c1, int skip0, int skip1, ff* re,
                                          ff* im, int step = 1) {
  float sr[4] = {0.f, 0.f, 0.f, 0.f}, cr[4] = {0.f, 0.f, 0.f, 0.f};
  float si[4] = {0.f, 0.f, 0.f, 0.f}, ci[4] = {0.f, 0.f, 0.f, 0.f};
  auto acc = [](float& sum, float& comp, float x, float y) {
    const float pr = __fmul_rn(x, y);
    const float pe = fmaf(x, y, -pr);  // x y = pr + pe exactly
    const ff t = two_sum(sum, pr);
    sum = t.hi;
    comp = __fadd_rn(comp, __fadd_rn(t.lo, pe));
  };
  for (int c = c0; c < c1; c += 4 * step) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int cc = c + u * step;
      float2 za = make_float2(0.f, 0.f), zb = make_float2(0.f, 0.f);
      if (cc < c1 && (cc < skip0 || cc >= skip1)) {
        za = zget(ra, cc);
        zb = zget(rb, cc);
      }
      acc(sr[u], cr[u], za.x, zb.x);
      acc(sr[u], cr[u], za.y, zb.y);
      acc(si[u], ci[u], za.y, zb.x);
      acc(si[u], ci[u], -za.x, zb.y);
    }
  }
  ff R = fast_two_sum(sr[0], cr[0]), I = fast_two_sum(si[0], ci[0]);
#pragma unroll
  for (int u = 1; u < 4; ++u) {
    R = ff_add(R, fast_two_sum(sr[u], cr[u]));
    I = ff_add(I, fast_two_sum(si[u], ci[u]));
  }
  *re = R;
  *im = I;
}

// S3a: upper triangle of Q_r = sigma^2 I + sum over streams other than the
// user's own of z z^H (sigma^2 = 1 after normalisation).  zget(row, col).
// Entries of z z^H summed over many streams can be far larger than the
// noise term (about 1e6 against 1 for a cell-centre user of the seven-cell
// layout), where FP32 rounding of the sum would blur the noise floor that
// eq. (9) resolves; so each entry is a compensated dot product (cov_entry),
// stored as a high part (sQ, read by the FP32 solves) and a low part
// (sQ + CK np, read by the FP64 and float-float solves).
// Four consecutive lanes share an entry (columns g, g + 4, ... for lane g)
// and add their parts by two exchanges, so that all warps take part.
template <class ZGet>
__device__ __forceinline__ void covariance_phase(const InstDesc& D, const Layout& Ly, ZGet zget, float2* sQ) {
  const int Nr = D.Nr, K = D.K, d = D.d, n = Ly.n, Cn = Ly.Cn, np = Ly.np, items = Ly.CK * np;
  float2* sQlo = sQ + Ly.CK * np;
  for (int base = 0; base < 4 * items; base += blockDim.x) {  // warp-uniform trip count (the exchanges)
    const int w = base + (int)threadIdx.x;
    const int e = w >> 2, g = w & 3;
    const bool act = e < items;
    const int r = act ? e / np : 0;
    int q = act ? e - r * np : 0, a = 0;
    while (q >= Nr - a) {
      q -= Nr - a;
      ++a;
    }
    const int bb = a + q;
    const int own0 = (r / K) * n + (r % K) * d;
    ff re = ff_from(0.f), im = ff_from(0.f);
    if (act) cov_entry(zget, r * Nr + a, r * Nr + bb, g, Cn, own0, own0 + d, &re, &im, 4);
    re = ff_add(re, ff_shfl_xor(re, 1));
    im = ff_add(im, ff_shfl_xor(im, 1));
    re = ff_add(re, ff_shfl_xor(re, 2));
    im = ff_add(im, ff_shfl_xor(im, 2));
    if (act && g == 0) {
      if (a == bb) re = ff_add(re, ff_from(1.f));
      sQ[e] = make_float2(re.hi, im.hi);
      sQlo[e] = make_float2(re.lo, im.lo);
    }
  }
}

struct NoIdle {
  __device__ void operator()() const {}
};

// S3b/S4: the per-user solves (eight lanes per user in FP64 or float-float,
// four in FP32), writing U, U W and the rates R_r (0 when want_ld is false
// and the rates are skipped); rho_sum_ff / rho_sum_exact sum them.  The own-stream block of user r is rows r Nr.., columns
// own0.. of Z (row stride ldz).  Zown: when non-null, the users' own-stream blocks in compact form (user r
// at Zown + r Nr d, row stride d), read instead of Z.  idle(): run by the
// warps that hold no user (all of their lanes), before the closing barrier;
// it must not use block-wide barriers.
template <class T, class Idle = NoIdle>
__device__ __forceinline__ void solve_phase(const InstDesc& D, const Layout& Ly, const float2* Z, int ldz,
                                              const float2* sQ, float2* sU, float2* sUW, double* sRho,
                                              const float* alpha_u, bool want_u, bool want_ld, double* red,
                                              int* fail, const float2* Zown = nullptr, Idle idle = Idle(),
                                              int r0 = 0, int nusers = -1) {
  const int Nr = D.Nr, K = D.K, d = D.d, n = Ly.n, np = Ly.np, CK = Ly.CK;
  const int NU = nusers < 0 ? CK : nusers;  // users r0 .. r0 + NU - 1 are solved
  // An FP64 warp instruction costs the same however few of its lanes are
  // active (on this part about 64 cycles for one warp, and one per 19 cycles
  // for the whole SM), so the users are packed densely: FP64 solves take
  // eight lanes per user (column x real/imaginary part, small_solve_pair),
  // FP32 solves four (column).  The trip count is warp-uniform (the solve
  // shuffles).
  constexpr bool kPair = !std::is_same<T, float>::value;  // FP64 or float-float: eight lanes per user
  constexpr int kLanes = kPair ? 8 : 4;
  bool had_user = false;
  for (int base = 0; base < kLanes * NU; base += blockDim.x) {
    const int e = base + threadIdx.x;
    const bool act = e < kLanes * NU;
    const int r = r0 + (act ? e / kLanes : 0), c = e & 3, ri = (e / 4) & (kLanes / 4 - 1);
    if (!__any_sync(0xffffffffu, act)) continue;  // warps without a user skip the solve
    had_user = true;
    const int own0 = Zown ? 0 : (r / K) * n + (r % K) * d;
    const float2* zr = Zown ? Zown + r * Nr * d : Z + (long long)r * Nr * ldz;
    const int ldr = Zown ? d : ldz;
    double ld = 0.0;
    bool ok;
    if constexpr (kPair)
      ok = small_solve_pair_dispatch<PairArith<T>>(Nr, d, c, ri, act, sQ + r * np, sQ + (CK + r) * np, zr, ldr,
                                                   own0, sU + r * Nr * d, sUW + r * Nr * d, &ld, want_u, want_ld);
    else
      ok = small_solve_dispatch<T>(Nr, d, c, act, sQ + r * np, zr, ldr, own0, sU + r * Nr * d, sUW + r * Nr * d,
                                   &ld, want_u, want_ld);
    if (act && c == 0 && ri == 0) {
      if (!ok || !isfinite(ld)) atomicExch(fail, kNumeric);
      sRho[r] = ok ? ld : 0.0;
    }
  }
  if (!had_user) idle();
  __syncthreads();
}

// rho = sum alpha_r R_r over the users (block-uniform).  In the iterations
// it only feeds the stage and stopping tests and the state returned by
// amm_get_state, so it is summed in float-float (about 1e-14 relative here,
// far below the FP32 rounding of the Z it comes from) without FP64
// instructions; the final WSR evaluation sums it in FP64.  The float-float
// scratch sits past the FP64 scratch of block_sum in `red`.  Both contain
// __syncthreads().
__device__ __forceinline__ ff rho_sum_ff(const double* sRho, const float* alpha_u, int CK, double* red) {
  ff part = ff_from(0.f);
  for (int r = threadIdx.x; r < CK; r += blockDim.x) part = ff_add(part, ff_mul(ff_from_double(sRho[r]), ff_from(alpha_u[r])));
  return block_sum_ff(part, reinterpret_cast<float*>(red) + 80);
}
__device__ __forceinline__ double rho_sum_exact(const double* sRho, const float* alpha_u, int CK, double* red) {
  double part = 0.0;
  for (int r = threadIdx.x; r < CK; r += blockDim.x) part += (double)alpha_u[r] * sRho[r];
  return block_sum(part, red);
}

// S6: Y_r = 2 alpha_r P_r (U_r^H zhat_r - S_r) for every user r and stream
// column c; sink(r, c, y) receives y[a] = Y[r Nr + a][c] for the Nr rows of r.
// tpu consecutive threads share a user: each keeps U_r and P_r in registers
// and takes every tpu-th column.
template <class ZGet, class Sink>
__device__ __forceinline__ void gradient_rhs_phase(const InstDesc& D, const Layout& Ly, ZGet zhat,
                                                   const float2* sU, const float2* sP, const float* alpha_u,
                                                   Sink sink, int cbeg = 0, int cend = -1) {
  const int Nr = D.Nr, K = D.K, d = D.d, n = Ly.n, CK = Ly.CK;
  const int Cn = cend < 0 ? Ly.Cn : cend;  // columns cbeg .. Cn - 1 (global numbering)
  const int ncol = Cn - cbeg;
  int tpu = (int)blockDim.x / CK;
  if (tpu < 1) tpu = 1;
  if (tpu > ncol) tpu = ncol;
  const int upp = (int)blockDim.x / tpu;  // users per pass
  const int rr = (int)threadIdx.x / tpu, c0 = (int)threadIdx.x - rr * tpu;
  for (int r = rr; rr < upp && r < CK; r += upp) {
    const int own0 = (r / K) * n + (r % K) * d;
    float2 Ur[kMaxNr][kMaxNr], Pr[kMaxNr][kMaxNr];
#pragma unroll
    for (int a = 0; a < kMaxNr; ++a)
#pragma unroll
      for (int s = 0; s < kMaxNr; ++s)
        if (a < Nr && s < d) {
          Ur[a][s] = sU[(r * Nr + a) * d + s];
          Pr[a][s] = sP[(r * Nr + a) * d + s];
        }
    const float sc2 = 2.f * alpha_u[r];
    for (int c = cbeg + c0; c < Cn; c += tpu) {
      float2 zh[kMaxNr];
#pragma unroll
      for (int a = 0; a < kMaxNr; ++a)
        if (a < Nr) zh[a] = zhat(r * Nr + a, c);
      float2 ts[kMaxNr];
#pragma unroll
      for (int s = 0; s < kMaxNr; ++s) {
        if (s < d) {
          float2 acc = make_float2((c - own0 == s) ? -1.f : 0.f, 0.f);
#pragma unroll
          for (int a = 0; a < kMaxNr; ++a)
            if (a < Nr) acc = cjfma(Ur[a][s], zh[a], acc);
          ts[s] = acc;
        }
      }
      float2 y[kMaxNr];
#pragma unroll
      for (int a = 0; a < kMaxNr; ++a) {
        float2 acc = make_float2(0.f, 0.f);
        if (a < Nr) {
#pragma unroll
          for (int s = 0; s < kMaxNr; ++s)
            if (s < d) acc = cfma(Pr[a][s], ts[s], acc);
        }
        y[a] = cscale(acc, sc2);
      }
      sink(r, c, y);
    }
  }
}

// Stage test of Algorithm 3 and the stopping test, run by one thread.
// ctrl: [0] t, [1] stage, [2] stage_iter, [3] last_stage, [4] stop,
// [6] step flags (bit 0 spectral, bit 1 freeze gamma_c).
// Whether iteration it of a launch needs R^t = WSR(V^{t-1}): for the stage
// test (stage I), the tolerance test, and in the last iteration so that a
// restored state carries rho_prev; inside the latched stage II of a
// fixed-count run nothing reads it.
__device__ __forceinline__ bool need_rate(int stage, int mode, int it, int n_iters) {
  return stage != 2 || mode != kFixed || it + 1 == n_iters;
}

__device__ __forceinline__ void stage_logic(int* ctrl, ff rho, ff rho_prev, int mode, float eps1, float eps2,
                                            int switch_iter, int step_rule, int tc) {
  // |R^t - R^{t-1}| / R^{t-1} <= eps, tested as |R^t - R^{t-1}| <= eps |R^{t-1}| with the
  // difference in float-float and the comparison in FP32 (a decision can differ
  // from an exact one only within about 1e-7 of the threshold)
  const int t = ctrl[0];
  const bool have_prev = !isnan(rho_prev.hi);
  const float diff = fabsf(ff_add(rho, ff_neg(rho_prev)).hi), ref = fabsf(rho_prev.hi);
  int stop = 0;
  if (mode == kTolerance && ctrl[3] == 2 && have_prev && ref > 0.f && diff <= eps2 * ref) stop = 1;
  int stage = ctrl[1], si = ctrl[2];
  if (!stop) {
    if (stage == 1) {
      const bool go = (switch_iter >= 1) ? (t >= switch_iter) : (have_prev && ref > 0.f && diff <= eps1 * ref);
      if (go) {
        stage = 2;
        si = 0;
      }
    }
    si += 1;
    ctrl[1] = stage;
    ctrl[2] = si;
    const int spectral = (step_rule == 1) || (step_rule == 0 && si <= tc);
    ctrl[6] = spectral | ((step_rule == 0 && si == tc) ? 2 : 0);
  }
  ctrl[4] = stop;
}

}  // namespace amm
