// Differentiable unrolled A-MMMSE: T iterations of Algorithm 3 with the
// step of iteration t a parameter gamma_t (shared by the batch) and the stage
// schedule fixed (stage I before iteration switch_iter, stage II from it on),
// and a hand-written adjoint that returns the gradient of WSR(V^T) with
// respect to every gamma_t and to the channels H.
//
// One block per instance, single cell (C = 1), everything in shared memory.
// The forward pass keeps (V^{c-1}, V^c) at every ck-th iteration; the
// backward pass recomputes each segment of ck iterations from its checkpoint
// and runs the adjoint of the iteration backwards through it.  Complex
// matrices are FP32; the per-user Nr x Nr / d x d Hermitian solves are
// float-float (pairs of FP32), the log-det FP64.
//
// Gradients use the real-gradient convention for complex variables: for a
// real L and complex X, Xbar = dL/dRe(X) + i dL/dIm(X), so that
// dL = Re tr(Xbar^H dX).  With it, the adjoint of C = A B is
// Abar = Cbar B^H, Bbar = A^H Cbar, and the gradient of the WMMSE objective
// f (eq. (8)) in V is G = H^H Y with Y_r = 2 alpha_r U_r W_r (U_r^H Z_r - S_r)
// (eq. (14) in matrix-free form).  At the MMSE receiver and W = E^{-1},
// WSR(V) = sum_r alpha_r d - min_{U,W} f, so by the envelope theorem the
// WSR's gradient is -G in V and -Y V^H in H.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <new>
#include <string>

#include "../../include/amm.h"
#include "amm_device.cuh"

namespace amm {
namespace {

constexpr int kUThreads = 256;

// Byte offsets of the shared-memory buffers of one instance.
struct ULayout {
  int H, Va, Vb, Vh, G, B, A1, A2, A3, Hb, Z, Zh, Y, Yb, Zb, Zhb;
  int Ti, Tc, U, W, P, Ub, Pb, red, ld, total;
};

__host__ __device__ inline int u_take(int& off, int bytes) {
  const int o = off;
  off = (off + bytes + 15) & ~15;
  return o;
}

__host__ __device__ inline ULayout u_layout(int K, int Nt, int Nr, int d) {
  const int m = K * Nr, n = K * d, vb = Nt * n * 8, zb = m * n * 8, hb = m * Nt * 8;
  ULayout L;
  int off = 0;
  L.H = u_take(off, hb);
  L.Va = u_take(off, vb);
  L.Vb = u_take(off, vb);
  L.Vh = u_take(off, vb);
  L.G = u_take(off, vb);
  L.B = u_take(off, vb);
  L.A1 = u_take(off, vb);
  L.A2 = u_take(off, vb);
  L.A3 = u_take(off, vb);
  L.Hb = u_take(off, hb);
  L.Z = u_take(off, zb);
  L.Zh = u_take(off, zb);
  L.Y = u_take(off, zb);
  L.Yb = u_take(off, zb);
  L.Zb = u_take(off, zb);
  L.Zhb = u_take(off, zb);
  L.Ti = u_take(off, K * Nr * Nr * 8);
  L.Tc = u_take(off, K * Nr * Nr * 8);
  L.U = u_take(off, K * Nr * d * 8);
  L.W = u_take(off, K * d * d * 8);
  L.P = u_take(off, K * Nr * d * 8);
  L.Ub = u_take(off, K * Nr * d * 8);
  L.Pb = u_take(off, K * Nr * d * 8);
  L.red = u_take(off, 66 * 8);
  L.ld = u_take(off, K * 8);
  L.total = off;
  return L;
}

struct UParams {
  int batch, K, Nt, Nr, d, T, ck, nseg, switch_iter, extrapolate;
  const float2* H;        // batch x m x Nt (as given)
  const float* sigma2;    // batch x K
  const float* alpha;     // batch x K
  const float* P;         // batch
  const float2* V0;       // batch x Nt x n
  const float* gamma;     // T
  float2* ckpt;           // batch x (2 nseg + 1) x Nt x n
  float2* hist;           // batch x (ck + 2) x Nt x n
  double* wsr;            // batch, bits
  const double* wsr_bar;  // batch
  float* gamma_bar;       // batch x T
  float2* H_bar;          // batch x m x Nt
  int* status;            // batch
};

// Start offset of a lane's sweep over the n columns of rows read with
// stride n by consecutive lanes.  Without it the 8-byte words of a
// half-warp share banks whenever n is even (all of them when n is a
// multiple of 16); with it they fall in distinct banks for n a multiple of
// 16 and spread out otherwise.  Odd n needs no offset.
__device__ __forceinline__ int bank_rot(int n) { return (n & 1) ? 0 : (int)(threadIdx.x & 31) % n; }

// conj(a) b
__device__ __forceinline__ float2 cjmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}

struct UView {
  int K, Nt, Nr, d, m, n;
  float2 *H, *Z, *Zh, *Y, *G, *Ti, *Tc, *U, *W, *P;
  double* ld;  // per user: log det E_r
  const float* alpha;
};

// ---- float-float helpers on small row-major complex matrices (one thread):
// pairs of FP32 (amm_ff.cuh, about 48 significant bits) on the FP32 pipe,
// where one warp's chain of FP64 instructions would wait ~64 cycles each
struct Zc {
  ff x, y;
};
__device__ __forceinline__ Zc zmk(ff x, ff y) {
  Zc r;
  r.x = x;
  r.y = y;
  return r;
}
__device__ __forceinline__ Zc zmkf(float x, float y) { return zmk(ff_from(x), ff_from(y)); }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ ff ff_half(ff a) { return ff_make(0.5f * a.hi, 0.5f * a.lo); }  // exact
__device__ __forceinline__ Zc zld(float2 v) { return zmkf(v.x, v.y); }
__device__ __forceinline__ Zc zmul(Zc a, Zc b) {
  return zmk(ff_fma(a.x, b.x, ff_neg(ff_mul(a.y, b.y))), ff_fma(a.x, b.y, ff_mul(a.y, b.x)));
}
__device__ __forceinline__ Zc zcmul(Zc a, Zc b) {  // conj(a) b
  return zmk(ff_fma(a.x, b.x, ff_mul(a.y, b.y)), ff_fma(a.x, b.y, ff_neg(ff_mul(a.y, b.x))));
}
__device__ __forceinline__ Zc zadd(Zc a, Zc b) { return zmk(ff_add(a.x, b.x), ff_add(a.y, b.y)); }
__device__ __forceinline__ Zc zsub(Zc a, Zc b) { return zmk(ff_sub(a.x, b.x), ff_sub(a.y, b.y)); }
__device__ __forceinline__ Zc zscale(Zc a, ff s) { return zmk(ff_mul(a.x, s), ff_mul(a.y, s)); }
__device__ __forceinline__ float2 zst(Zc a) { return make_float2(a.x.hi, a.y.hi); }  // hi = the value rounded

// Cholesky A = L L^H of an n x n Hermitian matrix (lower triangle of A
// read); returns false on a non-positive pivot.  iL[j] = 1 / L_jj (a
// float-float rsqrt per pivot, no division), and the pivots L_jj^2 go to
// piv[j].
template <int n>
__device__ __forceinline__ bool z_chol(const Zc* A, Zc* L, ff* iL, ff* piv) {
#pragma unroll
  for (int j = 0; j < n; ++j) {
    ff dj = A[j * n + j].x;
    for (int k = 0; k < j; ++k)
      dj = ff_sub(dj, ff_fma(L[j * n + k].x, L[j * n + k].x, ff_mul(L[j * n + k].y, L[j * n + k].y)));
    if (!(dj.hi > 0.f) || !(dj.hi < INFINITY)) return false;
    const ff rj = ff_rsqrt(dj);
    iL[j] = rj;
    piv[j] = dj;
    L[j * n + j] = zmk(ff_mul(dj, rj), ff_from(0.f));
    for (int i = j + 1; i < n; ++i) {
      Zc s = A[i * n + j];
      for (int k = 0; k < j; ++k) s = zsub(s, zmul(L[i * n + k], zmk(L[j * n + k].x, ff_neg(L[j * n + k].y))));
      L[i * n + j] = zscale(s, rj);
    }
    for (int i = 0; i < j; ++i) L[i * n + j] = zmkf(0.f, 0.f);
  }
  return true;
}

// X = A^{-1} B for A = L L^H (n x n), B n x k, all row-major.
template <int n, int k>
__device__ __forceinline__ void z_chol_solve(const Zc* L, const ff* iL, const Zc* B, Zc* X) {
#pragma unroll
  for (int c = 0; c < k; ++c) {
    for (int i = 0; i < n; ++i) {  // L y = b
      Zc s = B[i * k + c];
      for (int j = 0; j < i; ++j) s = zsub(s, zmul(L[i * n + j], X[j * k + c]));
      X[i * k + c] = zscale(s, iL[i]);
    }
    for (int i = n - 1; i >= 0; --i) {  // L^H x = y
      Zc s = X[i * k + c];
      for (int j = i + 1; j < n; ++j) s = zsub(s, zcmul(L[j * n + i], X[j * k + c]));
      X[i * k + c] = zscale(s, iL[i]);
    }
  }
}

// Per-user solves of one iteration (thread r < K), from Z = H V^{t-1} and
// T_r = I + Z_r Z_r^H (all columns, FP32, in X.Tc): U_r = T_r^{-1} Z_own (eq. (9), sigma^2 = 1),
// E_r = I - U_r^H Z_own, W_r = E_r^{-1} (eq. (10); I in stage I), P_r = U_r W_r.
// Stores T_r^{-1}, U, W, P and log det E_r.  Returns false on a failed factorisation.
// Nr and d are compile-time, so the small matrices live in registers.
template <int NR, int DD>
__device__ __noinline__ bool u_solve_user_t(const UView& X, int r, bool stage2, bool want_ld) {
  constexpr int Nr = NR, d = DD;
  const int n = X.n;
  Zc A[16], L[16], I4[16], Ti[16], Zo[16], Uu[16], E[16], Le[16], Wm[16];
  for (int a = 0; a < Nr; ++a)
    for (int b = 0; b < Nr; ++b) {
      A[a * Nr + b] = zld(X.Tc[(r * Nr + a) * Nr + b]);  // FP32 covariance (u_forward_iter)
      I4[a * Nr + b] = zmkf(a == b ? 1.f : 0.f, 0.f);
    }
  ff iLt[4], pv[4];
  if (!z_chol<Nr>(A, L, iLt, pv)) return false;
  z_chol_solve<Nr, Nr>(L, iLt, I4, Ti);
  for (int a = 0; a < Nr; ++a)
    for (int s = 0; s < d; ++s) Zo[a * d + s] = zld(X.Z[(r * Nr + a) * n + r * d + s]);
  for (int a = 0; a < Nr; ++a)
    for (int s = 0; s < d; ++s) {
      Zc acc = zmkf(0.f, 0.f);
      for (int b = 0; b < Nr; ++b) acc = zadd(acc, zmul(Ti[a * Nr + b], Zo[b * d + s]));
      Uu[a * d + s] = acc;
    }
  for (int s = 0; s < d; ++s)
    for (int u = 0; u < d; ++u) {
      Zc acc = zmkf(s == u ? 1.f : 0.f, 0.f);
      for (int a = 0; a < Nr; ++a) acc = zsub(acc, zcmul(Uu[a * d + s], Zo[a * d + u]));
      E[s * d + u] = acc;
    }
  for (int s = 0; s < d; ++s)  // Hermitian part
    for (int u = s; u < d; ++u) {
      const Zc h = zmk(ff_half(ff_add(E[s * d + u].x, E[u * d + s].x)), ff_half(ff_sub(E[s * d + u].y, E[u * d + s].y)));
      E[s * d + u] = h;
      E[u * d + s] = zmk(h.x, ff_neg(h.y));
    }
  ff iLe[4], pe[4];
  if (!z_chol<d>(E, Le, iLe, pe)) return false;
  for (int s = 0; s < d; ++s)
    for (int u = 0; u < d; ++u) I4[s * d + u] = zmkf(s == u ? 1.f : 0.f, 0.f);
  if (stage2) {
    z_chol_solve<d, d>(Le, iLe, I4, Wm);
  } else {
    for (int q = 0; q < d * d; ++q) Wm[q] = I4[q];
  }
  for (int q = 0; q < Nr * Nr; ++q) X.Ti[r * Nr * Nr + q] = zst(Ti[q]);
  for (int q = 0; q < Nr * d; ++q) X.U[r * Nr * d + q] = zst(Uu[q]);
  for (int q = 0; q < d * d; ++q) X.W[r * d * d + q] = zst(Wm[q]);
  for (int a = 0; a < Nr; ++a)
    for (int s = 0; s < d; ++s) {
      Zc acc = zmkf(0.f, 0.f);
      for (int u = 0; u < d; ++u) acc = zadd(acc, zmul(Uu[a * d + u], Wm[u * d + s]));
      X.P[(r * Nr + a) * d + s] = zst(acc);
    }
  if (want_ld) {  // log det E_r from the pivots, only where the WSR is read (one FP64 log)
    ff prod = ff_from(1.f);
    for (int j = 0; j < d; ++j) prod = ff_mul(prod, pe[j]);
    X.ld[r] = log(ff_to_double(prod));
  }
  return true;
}

// One (N_r, d) pair per instantiation: N_r <= 4, d <= N_r.
#define AMM_U_PAIRS(F) F(1, 1) F(2, 1) F(2, 2) F(3, 1) F(3, 2) F(3, 3) F(4, 1) F(4, 2) F(4, 3) F(4, 4)

__device__ __forceinline__ bool u_solve_user(const UView& X, int r, bool stage2, bool want_ld) {
#define AMM_U_SOLVE(a, b) \
  if (X.Nr == a && X.d == b) return u_solve_user_t<a, b>(X, r, stage2, want_ld);
  AMM_U_PAIRS(AMM_U_SOLVE)
#undef AMM_U_SOLVE
  return false;
}

// Forward part of iteration t shared by both passes: Z = H Va, the per-user
// solves, Vh = Vhat, Zh = H Vhat, Y (eq. (14) form) and G = H^H Y.
__device__ void u_forward_iter(const UView& X, bool stage2, float omega, const float2* Va, const float2* Vb,
                               float2* Vh, int* fail, bool want_ld = false) {
  const int m = X.m, n = X.n, Nt = X.Nt, Nr = X.Nr, d = X.d, K = X.K;
  block_cgemm_tiled<0>(gemm_tile_for(0, m, n), m, n, Nt, X.H, Nt, Va, n,
                       [&](int r, int c, float2 v) { X.Z[r * n + c] = v; });
  for (int e = threadIdx.x; e < Nt * n; e += blockDim.x)
    Vh[e] = make_float2((1.f + omega) * Va[e].x - omega * Vb[e].x, (1.f + omega) * Va[e].y - omega * Vb[e].y);
  __syncthreads();
  // T_r = I + sum over all columns of z_a conj(z_b), one thread per entry (FP32).
  // Rows of Z are n apart, so each user sweeps the columns from its own
  // offset (the lanes of one user read the same addresses).
  for (int e = threadIdx.x; e < K * Nr * Nr; e += blockDim.x) {
    const int r = e / (Nr * Nr), ab = e - r * Nr * Nr, a = ab / Nr, b = ab - a * Nr;
    const int rot = (n & 1) ? 0 : r % n;
    float2 acc = make_float2(a == b ? 1.f : 0.f, 0.f);
    for (int k = 0; k < n; ++k) {
      const int c = (k + rot < n) ? k + rot : k + rot - n;
      acc = cjfma(X.Z[(r * Nr + b) * n + c], X.Z[(r * Nr + a) * n + c], acc);
    }
    X.Tc[e] = acc;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < K; r += blockDim.x)
    if (!u_solve_user(X, r, stage2, want_ld)) atomicExch(fail, kNumeric);
  block_cgemm_tiled<0>(gemm_tile_for(0, m, n), m, n, Nt, X.H, Nt, Vh, n,
                       [&](int r, int c, float2 v) { X.Zh[r * n + c] = v; });
  __syncthreads();
  // Y_r = 2 alpha_r P_r (U_r^H Zh_r - S_r), one thread per (user, column)
  for (int e = threadIdx.x; e < K * n; e += blockDim.x) {
    const int r = e / n, c = e - r * n;
    float2 As[kMaxNr];
    for (int s = 0; s < d; ++s) {
      float2 acc = make_float2(c == r * d + s ? -1.f : 0.f, 0.f);
      for (int b = 0; b < Nr; ++b) acc = cjfma(X.U[(r * Nr + b) * d + s], X.Zh[(r * Nr + b) * n + c], acc);
      As[s] = acc;
    }
    const float a2 = 2.f * X.alpha[r];
    for (int a = 0; a < Nr; ++a) {
      float2 acc = make_float2(0.f, 0.f);
      for (int s = 0; s < d; ++s) acc = cfma(X.P[(r * Nr + a) * d + s], As[s], acc);
      X.Y[(r * Nr + a) * n + c] = cscale(acc, a2);
    }
  }
  __syncthreads();
  block_cgemm_tiled<1>(gemm_tile_for(0, Nt, n), Nt, n, m, X.H, Nt, X.Y, n,
                       [&](int q, int c, float2 v) { X.G[q * n + c] = v; });
  __syncthreads();
}

__device__ __forceinline__ float u_omega(const UParams& p, int t) {
  return (p.extrapolate && t >= 3) ? (float)(t - 2) / (float)(t + 1) : 0.f;
}

__device__ __forceinline__ float2* u_ckpt(const UParams& p, int b, int slot) {
  const long long vn = (long long)p.Nt * p.K * p.d;
  return p.ckpt + ((long long)b * (2 * p.nseg + 1) + slot) * vn;
}

__device__ UView u_view(const UParams& p, unsigned char* smem, const ULayout& L, int b) {
  UView X;
  X.K = p.K;
  X.Nt = p.Nt;
  X.Nr = p.Nr;
  X.d = p.d;
  X.m = p.K * p.Nr;
  X.n = p.K * p.d;
  X.H = reinterpret_cast<float2*>(smem + L.H);
  X.Z = reinterpret_cast<float2*>(smem + L.Z);
  X.Zh = reinterpret_cast<float2*>(smem + L.Zh);
  X.Y = reinterpret_cast<float2*>(smem + L.Y);
  X.G = reinterpret_cast<float2*>(smem + L.G);
  X.Ti = reinterpret_cast<float2*>(smem + L.Ti);
  X.Tc = reinterpret_cast<float2*>(smem + L.Tc);
  X.U = reinterpret_cast<float2*>(smem + L.U);
  X.W = reinterpret_cast<float2*>(smem + L.W);
  X.P = reinterpret_cast<float2*>(smem + L.P);
  X.ld = reinterpret_cast<double*>(smem + L.ld);
  X.alpha = p.alpha + (long long)b * p.K;
  return X;
}

// H_n = H / sigma_r per user row
__device__ void u_load_h(const UParams& p, const UView& X, int b) {
  const float2* Hg = p.H + (long long)b * X.m * X.Nt;
  for (int e = threadIdx.x; e < X.m * X.Nt; e += blockDim.x) {
    const int i = e / X.Nt;
    const float is = rsqrtf(p.sigma2[(long long)b * X.K + i / X.Nr]);
    X.H[e] = cscale(Hg[e], is);
  }
}

// V^t = project(Vh - gamma G) into out; returns ||Vh - gamma G||^2
__device__ double u_step_project(const UView& X, float gam, float Pc, const float2* Vh, float2* out, double* red) {
  const int N = X.Nt * X.n;
  ff sf = ff_from(0.f);  // float-float with exact products: no FP64 instruction per element
  for (int e = threadIdx.x; e < N; e += blockDim.x) {
    const float2 v = make_float2(Vh[e].x - gam * X.G[e].x, Vh[e].y - gam * X.G[e].y);
    sf = ff_dot_acc(ff_dot_acc(sf, v.x, v.x), v.y, v.y);
  }
  sf = block_sum_ff(sf, reinterpret_cast<float*>(red) + 80);
  const double s = ff_to_double(sf);
  const float sc = (sf.hi > Pc) ? sqrtf(Pc / sf.hi) : 1.f;
  for (int e = threadIdx.x; e < N; e += blockDim.x)
    out[e] = make_float2((Vh[e].x - gam * X.G[e].x) * sc, (Vh[e].y - gam * X.G[e].y) * sc);
  __syncthreads();
  return s;
}

__global__ void __launch_bounds__(kUThreads) u_forward_kernel(UParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_fail;
  const int b = blockIdx.x;
  const ULayout L = u_layout(p.K, p.Nt, p.Nr, p.d);
  const UView X = u_view(p, smem, L, b);
  double* red = reinterpret_cast<double*>(smem + L.red);
  if (threadIdx.x == 0) s_fail = kOk;
  float2* Vbuf[3] = {reinterpret_cast<float2*>(smem + L.Va), reinterpret_cast<float2*>(smem + L.Vb),
                     reinterpret_cast<float2*>(smem + L.B)};
  float2* Vh = reinterpret_cast<float2*>(smem + L.Vh);
  const int N = X.Nt * X.n;
  u_load_h(p, X, b);
  const float2* V0 = p.V0 + (long long)b * N;
  for (int e = threadIdx.x; e < N; e += blockDim.x) Vbuf[0][e] = Vbuf[1][e] = V0[e];
  __syncthreads();
  const float Pc = p.P[b];
  int ia = 0, ib = 1, in = 2;  // V^{t-1}, V^{t-2}, free
  for (int t = 1; t <= p.T; ++t) {
    if ((t - 1) % p.ck == 0) {
      const int sgi = (t - 1) / p.ck;
      float2* c0 = u_ckpt(p, b, 2 * sgi);
      float2* c1 = u_ckpt(p, b, 2 * sgi + 1);
      for (int e = threadIdx.x; e < N; e += blockDim.x) {
        c0[e] = Vbuf[ib][e];
        c1[e] = Vbuf[ia][e];
      }
    }
    const bool stage2 = p.switch_iter >= 1 && t >= p.switch_iter;
    u_forward_iter(X, stage2, u_omega(p, t), Vbuf[ia], Vbuf[ib], Vh, &s_fail);
    u_step_project(X, p.gamma[t - 1], Pc, Vh, Vbuf[in], red);
    const int old_b = ib;
    ib = ia;
    ia = in;
    in = old_b;
  }
  // V^T and WSR(V^T) = sum_r alpha_r log det E_r^{-1} at the MMSE receiver
  float2* cT = u_ckpt(p, b, 2 * p.nseg);
  for (int e = threadIdx.x; e < N; e += blockDim.x) cT[e] = Vbuf[ia][e];
  u_forward_iter(X, true, 0.f, Vbuf[ia], Vbuf[ia], Vh, &s_fail, true);
  double part = 0.0;
  for (int r = threadIdx.x; r < X.K; r += blockDim.x) part += (double)X.alpha[r] * (-X.ld[r]);
  const double w = block_sum(part, red);
  if (threadIdx.x == 0) {
    p.wsr[b] = w / 0.69314718055994530942;
    p.status[b] = s_fail;
  }
}

// Per-user part of the adjoint of one iteration (one warp per user r, its
// lanes over the columns): Abar = 2 alpha P^H Ybar, Ubar, Pbar (summed over
// the lanes) and Zhbar = U Abar over the columns, then (every lane) the
// adjoints of P = U W, W = E^{-1}, E = I - U^H Zo, U = T^{-1} Zo and
// T = I + Z Z^H, giving Zbar_r.  N_r and d are compile-time, so the small
// matrices live in registers.
template <int NR, int DD>
__device__ __noinline__ void u_adjoint_user_t(const UView& X, int r, bool stage2, const float2* Yb, float2* Zhb,
                                                 float2* Zb, float2* Ub, float2* Pb) {
  constexpr int Nr = NR, d = DD;
  const int n = X.n, lane = threadIdx.x & 31;
  const float a2 = 2.f * X.alpha[r];
  float2 ub[16], pb[16], Ur[16], Pr[16];
#pragma unroll
  for (int q = 0; q < Nr * d; ++q) {
    ub[q] = pb[q] = make_float2(0.f, 0.f);
    Ur[q] = X.U[r * Nr * d + q];
    Pr[q] = X.P[r * Nr * d + q];
  }
  // the warp's lanes take the columns: A = U^H Zh - S, Abar = 2 alpha P^H Ybar
  for (int c = lane; c < n; c += 32) {
    float2 As[kMaxNr], Ab[kMaxNr];
#pragma unroll
    for (int s2 = 0; s2 < d; ++s2) {
      float2 acc = make_float2(c == r * d + s2 ? -1.f : 0.f, 0.f);
      float2 acb = make_float2(0.f, 0.f);
#pragma unroll
      for (int a = 0; a < Nr; ++a) {
        acc = cjfma(Ur[a * d + s2], X.Zh[(r * Nr + a) * n + c], acc);
        acb = cjfma(Pr[a * d + s2], Yb[(r * Nr + a) * n + c], acb);
      }
      As[s2] = acc;
      Ab[s2] = cscale(acb, a2);
    }
#pragma unroll
    for (int a = 0; a < Nr; ++a) {
      const float2 zh = X.Zh[(r * Nr + a) * n + c], yb = Yb[(r * Nr + a) * n + c];
      float2 zhb = make_float2(0.f, 0.f);
#pragma unroll
      for (int s2 = 0; s2 < d; ++s2) {
        // Ubar += Zh Abar^H;  Pbar += 2 alpha Ybar A^H;  Zhbar = U Abar
        ub[a * d + s2] = cfma(zh, make_float2(Ab[s2].x, -Ab[s2].y), ub[a * d + s2]);
        pb[a * d + s2] = cfma(cscale(yb, a2), make_float2(As[s2].x, -As[s2].y), pb[a * d + s2]);
        zhb = cfma(Ur[a * d + s2], Ab[s2], zhb);
      }
      Zhb[(r * Nr + a) * n + c] = zhb;
    }
  }
  // the column sums of Ubar and Pbar over the lanes; every lane holds them
#pragma unroll
  for (int q = 0; q < Nr * d; ++q) {
    ub[q] = warp_sum(ub[q]);
    pb[q] = warp_sum(pb[q]);
  }
  // From here FP32: products of the small matrices that the float-float
  // forward solve produced (no factorisation).  P = U W: Ubar += Pbar W^H, Wbar = U^H Pbar
  float2 Ubr[16], Wb[16], Uu[16], Wm[16], Eb[16], Bm[16], Tb[16], Ti[16];
  for (int q = 0; q < Nr * d; ++q) Uu[q] = X.U[r * Nr * d + q];
  for (int q = 0; q < d * d; ++q) Wm[q] = X.W[r * d * d + q];
  for (int q = 0; q < Nr * Nr; ++q) Ti[q] = X.Ti[r * Nr * Nr + q];
  for (int a = 0; a < Nr; ++a)
    for (int s2 = 0; s2 < d; ++s2) {
      float2 acc = ub[a * d + s2];
      for (int u = 0; u < d; ++u) acc = cadd(acc, cmul(pb[a * d + u], make_float2(Wm[s2 * d + u].x, -Wm[s2 * d + u].y)));
      Ubr[a * d + s2] = acc;
    }
  for (int q = 0; q < d * d; ++q) Eb[q] = make_float2(0.f, 0.f);
  if (stage2) {
    for (int s2 = 0; s2 < d; ++s2)
      for (int u = 0; u < d; ++u) {
        float2 acc = make_float2(0.f, 0.f);
        for (int a = 0; a < Nr; ++a) acc = cadd(acc, cjmul(Uu[a * d + s2], pb[a * d + u]));
        Wb[s2 * d + u] = acc;
      }
    // W = E^{-1}: Ebar = -W^H Wbar W^H  (W Hermitian)
    float2 tmp[16];
    for (int s2 = 0; s2 < d; ++s2)
      for (int u = 0; u < d; ++u) {
        float2 acc = make_float2(0.f, 0.f);
        for (int v = 0; v < d; ++v) acc = cadd(acc, cmul(Wm[s2 * d + v], Wb[v * d + u]));
        tmp[s2 * d + u] = acc;
      }
    for (int s2 = 0; s2 < d; ++s2)
      for (int u = 0; u < d; ++u) {
        float2 acc = make_float2(0.f, 0.f);
        for (int v = 0; v < d; ++v) acc = cadd(acc, cmul(tmp[s2 * d + v], Wm[v * d + u]));
        Eb[s2 * d + u] = make_float2(-acc.x, -acc.y);
      }
    // E = I - U^H Zo: Ubar += -Zo Ebar^H
    for (int a = 0; a < Nr; ++a)
      for (int s2 = 0; s2 < d; ++s2) {
        float2 acc = Ubr[a * d + s2];
        for (int u = 0; u < d; ++u) {
          const float2 zo = X.Z[(r * Nr + a) * n + r * d + u];
          acc = csub(acc, cmul(zo, make_float2(Eb[s2 * d + u].x, -Eb[s2 * d + u].y)));
        }
        Ubr[a * d + s2] = acc;
      }
  }
  // U = T^{-1} Zo: Bm = T^{-1} Ubar; Zo-bar += Bm; Tbar = -Bm U^H
  for (int a = 0; a < Nr; ++a)
    for (int s2 = 0; s2 < d; ++s2) {
      float2 acc = make_float2(0.f, 0.f);
      for (int c2 = 0; c2 < Nr; ++c2) acc = cadd(acc, cmul(Ti[a * Nr + c2], Ubr[c2 * d + s2]));
      Bm[a * d + s2] = acc;
    }
  for (int a = 0; a < Nr; ++a)
    for (int c2 = 0; c2 < Nr; ++c2) {
      float2 acc = make_float2(0.f, 0.f);
      for (int s2 = 0; s2 < d; ++s2) acc = csub(acc, cmul(Bm[a * d + s2], make_float2(Uu[c2 * d + s2].x, -Uu[c2 * d + s2].y)));
      Tb[a * Nr + c2] = acc;
    }
  // T = I + Z Z^H: Zbar_r = (Tbar + Tbar^H) Z_r (FP32 over the columns);
  // own columns also get Bm - U Ebar
  float2 sym[16], ownb[16];
  for (int a = 0; a < Nr; ++a)
    for (int c2 = 0; c2 < Nr; ++c2)
      sym[a * Nr + c2] = make_float2(Tb[a * Nr + c2].x + Tb[c2 * Nr + a].x, Tb[a * Nr + c2].y - Tb[c2 * Nr + a].y);
  for (int a = 0; a < Nr; ++a)
    for (int s2 = 0; s2 < d; ++s2) {
      float2 acc = Bm[a * d + s2];
      for (int u = 0; u < d; ++u) acc = csub(acc, cmul(Uu[a * d + u], Eb[u * d + s2]));
      ownb[a * d + s2] = acc;
    }
  for (int c = lane; c < n; c += 32) {
    const bool own = c >= r * d && c < r * d + d;
    for (int a = 0; a < Nr; ++a) {
      float2 acc = make_float2(0.f, 0.f);
      if (own)
#pragma unroll
        for (int u = 0; u < d; ++u)
          if (c - r * d == u) acc = ownb[a * d + u];  // constant index: ownb stays in registers
      for (int c2 = 0; c2 < Nr; ++c2) acc = cfma(sym[a * Nr + c2], X.Z[(r * Nr + c2) * n + c], acc);
      Zb[(r * Nr + a) * n + c] = acc;
    }
  }
  if (lane == 0)
    for (int q = 0; q < Nr * d; ++q) {
      Ub[r * Nr * d + q] = Ubr[q];
      Pb[r * Nr * d + q] = pb[q];
    }
}

__device__ __forceinline__ void u_adjoint_user(const UView& X, int r, bool stage2, const float2* Yb, float2* Zhb,
                                               float2* Zb, float2* Ub, float2* Pb) {
#define AMM_U_ADJ(a, b) \
  if (X.Nr == a && X.d == b) return u_adjoint_user_t<a, b>(X, r, stage2, Yb, Zhb, Zb, Ub, Pb);
  AMM_U_PAIRS(AMM_U_ADJ)
#undef AMM_U_ADJ
}

// Adjoint of one iteration t.  In: A1 = Vbar^t (complete), A2 = the part of
// Vbar^{t-1} already collected.  Out: A2 += this iteration's share of
// Vbar^{t-1}, A3 = its share of Vbar^{t-2}, Hb += its share of Hbar,
// gamma_bar[t-1].
__device__ void u_adjoint_iter(const UParams& p, const UView& X, const ULayout& L, unsigned char* smem, int b, int t,
                               const float2* Va, const float2* Vb, const float2* A1, float2* A2, float2* A3,
                               int* fail) {
  const int m = X.m, n = X.n, Nt = X.Nt, K = X.K, N = Nt * n;
  double* red = reinterpret_cast<double*>(smem + L.red);
  float2* Vh = reinterpret_cast<float2*>(smem + L.Vh);
  float2* B = reinterpret_cast<float2*>(smem + L.B);
  float2* Hb = reinterpret_cast<float2*>(smem + L.Hb);
  float2* Yb = reinterpret_cast<float2*>(smem + L.Yb);
  float2* Zb = reinterpret_cast<float2*>(smem + L.Zb);
  float2* Zhb = reinterpret_cast<float2*>(smem + L.Zhb);
  float2* Ub = reinterpret_cast<float2*>(smem + L.Ub);
  float2* Pb = reinterpret_cast<float2*>(smem + L.Pb);
  const bool stage2 = p.switch_iter >= 1 && t >= p.switch_iter;
  const float omega = u_omega(p, t);
  const float gam = p.gamma[t - 1];
  const float Pc = p.P[b];
  u_forward_iter(X, stage2, omega, Va, Vb, Vh, fail);
  // projection: Vt = Vh - gam G, V^t = c Vt with c = sqrt(P / ||Vt||^2) when active
  // the sums in float-float with exact products (no FP64 instruction per element)
  float* redf = reinterpret_cast<float*>(red) + 80;
  ff s = ff_from(0.f), ip = ff_from(0.f);
  for (int e = threadIdx.x; e < N; e += blockDim.x) {
    const float2 v = make_float2(Vh[e].x - gam * X.G[e].x, Vh[e].y - gam * X.G[e].y);
    s = ff_dot_acc(ff_dot_acc(s, v.x, v.x), v.y, v.y);
    ip = ff_dot_acc(ff_dot_acc(ip, A1[e].x, v.x), A1[e].y, v.y);
  }
  s = block_sum_ff(s, redf);
  ip = block_sum_ff(ip, redf);
  const bool active = s.hi > Pc;
  const float cc = active ? sqrtf(Pc / s.hi) : 1.f;
  const float kk = active ? ip.hi / s.hi : 0.f;
  ff gb = ff_from(0.f);
  for (int e = threadIdx.x; e < N; e += blockDim.x) {
    const float2 v = make_float2(Vh[e].x - gam * X.G[e].x, Vh[e].y - gam * X.G[e].y);
    const float2 bt = make_float2(cc * (A1[e].x - kk * v.x), cc * (A1[e].y - kk * v.y));  // Vtilde-bar
    B[e] = bt;
    gb = ff_dot_acc(ff_dot_acc(gb, bt.x, X.G[e].x), bt.y, X.G[e].y);
  }
  gb = block_sum_ff(gb, redf);  // also orders the writes of B before the reads below
  if (threadIdx.x == 0) p.gamma_bar[(long long)b * p.T + (t - 1)] = -gb.hi;
  // Gbar = -gam B;  Ybar = H Gbar
  block_cgemm_tiled<0>(gemm_tile_for(0, m, n), m, n, Nt, X.H, Nt, B, n,
                       [&](int r, int c, float2 v) { Yb[r * n + c] = cscale(v, -gam); });
  __syncthreads();
  // per user: Abar = 2 alpha P^H Ybar, Ubar, Pbar, Zhbar = U Abar; then W, E and T
  // one warp per user (lanes over the columns)
  for (int r = threadIdx.x >> 5; r < K; r += blockDim.x >> 5) u_adjoint_user(X, r, stage2, Yb, Zhb, Zb, Ub, Pb);
  __syncthreads();
  // Hbar += Y Gbar^H + Zhbar Vhat^H + Zbar Va^H  (Gbar = -gam B): a sum over
  // 3 n products per entry, 2 x 4 entries per thread (rows i0 + a ntr,
  // columns q0 + b ntc), the 3 x 6 operand values of a column loaded once
  // for the 24 products.  Rows q n of B, Vhat, Va are n apart, so each lane
  // starts its column sweep at its own offset (bank_rot).
  {
    const int rot = bank_rot(n);
    constexpr int TM = 2, TN = 4;
    const int ntr = (m + TM - 1) / TM, ntc = (Nt + TN - 1) / TN;
    for (int tile = threadIdx.x; tile < ntr * ntc; tile += blockDim.x) {
      const int tr = tile / ntc, tq = tile - tr * ntc;
      int ii[TM], qq[TN];
#pragma unroll
      for (int a = 0; a < TM; ++a) ii[a] = min(tr + a * ntr, m - 1);
#pragma unroll
      for (int bq = 0; bq < TN; ++bq) qq[bq] = min(tq + bq * ntc, Nt - 1);
      float2 acc[TM][TN];
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int bq = 0; bq < TN; ++bq) acc[a][bq] = make_float2(0.f, 0.f);
      for (int k = 0; k < n; ++k) {
        const int c = (k + rot < n) ? k + rot : k + rot - n;
        float2 y[TM], zh[TM], zb[TM], g[TN], vh[TN], va[TN];
#pragma unroll
        for (int a = 0; a < TM; ++a) {
          y[a] = X.Y[ii[a] * n + c];
          zh[a] = Zhb[ii[a] * n + c];
          zb[a] = Zb[ii[a] * n + c];
        }
#pragma unroll
        for (int bq = 0; bq < TN; ++bq) {
          const float2 gb = cscale(B[qq[bq] * n + c], -gam);
          g[bq] = make_float2(gb.x, -gb.y);
          vh[bq] = make_float2(Vh[qq[bq] * n + c].x, -Vh[qq[bq] * n + c].y);
          va[bq] = make_float2(Va[qq[bq] * n + c].x, -Va[qq[bq] * n + c].y);
        }
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
          for (int bq = 0; bq < TN; ++bq)
            acc[a][bq] = cfma(zb[a], va[bq], cfma(zh[a], vh[bq], cfma(y[a], g[bq], acc[a][bq])));
      }
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int bq = 0; bq < TN; ++bq) {
          const int i = tr + a * ntr, q = tq + bq * ntc;
          if (i < m && q < Nt) Hb[i * Nt + q] = cadd(Hb[i * Nt + q], acc[a][bq]);
        }
    }
  }
  __syncthreads();
  // Vhat-bar = B + H^H Zhbar (in B);  A2 += H^H Zbar + (1 + w) Vhat-bar;  A3 = -w Vhat-bar
  block_cgemm_tiled<1>(gemm_tile_for(0, Nt, n), Nt, n, m, X.H, Nt, Zhb, n,
                       [&](int q, int c, float2 v) { B[q * n + c] = cadd(B[q * n + c], v); });
  __syncthreads();
  block_cgemm_tiled<1>(gemm_tile_for(0, Nt, n), Nt, n, m, X.H, Nt, Zb, n, [&](int q, int c, float2 zz) {
    const int e = q * n + c;
    const float2 vhb = B[e];
    A2[e] = make_float2(A2[e].x + zz.x + (1.f + omega) * vhb.x, A2[e].y + zz.y + (1.f + omega) * vhb.y);
    A3[e] = make_float2(-omega * vhb.x, -omega * vhb.y);
  });
  __syncthreads();
}

__global__ void __launch_bounds__(kUThreads) u_backward_kernel(UParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_fail;
  const int b = blockIdx.x;
  const ULayout L = u_layout(p.K, p.Nt, p.Nr, p.d);
  const UView X = u_view(p, smem, L, b);
  if (threadIdx.x == 0) s_fail = kOk;
  const int N = X.Nt * X.n;
  u_load_h(p, X, b);
  float2* Vh = reinterpret_cast<float2*>(smem + L.Vh);
  float2* Va = reinterpret_cast<float2*>(smem + L.Va);
  float2* Vb = reinterpret_cast<float2*>(smem + L.Vb);
  float2* Acc[3] = {reinterpret_cast<float2*>(smem + L.A1), reinterpret_cast<float2*>(smem + L.A2),
                    reinterpret_cast<float2*>(smem + L.A3)};
  float2* Hb = reinterpret_cast<float2*>(smem + L.Hb);
  double* red = reinterpret_cast<double*>(smem + L.red);
  const double wb = p.wsr_bar[b] / 0.69314718055994530942;  // dL / dWSR in nats
  // WSR(V^T): Vbar^T = -wb G*, Hbar = -wb Y* (V^T)^H at the MMSE receiver and W = E^{-1}
  const float2* cT = u_ckpt(p, b, 2 * p.nseg);
  for (int e = threadIdx.x; e < N; e += blockDim.x) Va[e] = cT[e];
  __syncthreads();
  u_forward_iter(X, true, 0.f, Va, Va, Vh, &s_fail);
  const float wf = (float)wb;
  for (int e = threadIdx.x; e < N; e += blockDim.x) {
    Acc[0][e] = cscale(X.G[e], -wf);
    Acc[1][e] = make_float2(0.f, 0.f);
  }
  const int rot = bank_rot(X.n);
  for (int e = threadIdx.x; e < X.m * X.Nt; e += blockDim.x) {
    const int i = e / X.Nt, q = e - i * X.Nt;
    float2 acc = make_float2(0.f, 0.f);
    for (int k = 0; k < X.n; ++k) {
      const int c = (k + rot < X.n) ? k + rot : k + rot - X.n;
      acc = cfma(X.Y[i * X.n + c], make_float2(Va[q * X.n + c].x, -Va[q * X.n + c].y), acc);
    }
    Hb[e] = cscale(acc, -wf);
  }
  __syncthreads();
  const long long vn = (long long)N;
  float2* hist = p.hist + (long long)b * (p.ck + 2) * vn;  // hist[j] = V^{c0 - 1 + j}
  for (int sg = p.nseg - 1; sg >= 0; --sg) {
    const int c0 = sg * p.ck, c1 = min(c0 + p.ck, p.T);
    const float2* k0 = u_ckpt(p, b, 2 * sg);
    const float2* k1 = u_ckpt(p, b, 2 * sg + 1);
    for (int e = threadIdx.x; e < N; e += blockDim.x) {
      Vb[e] = hist[e] = k0[e];
      Va[e] = hist[vn + e] = k1[e];
    }
    __syncthreads();
    // recompute V^{c0+1} .. V^{c1-1} into hist
    for (int t = c0 + 1; t < c1; ++t) {
      const bool stage2 = p.switch_iter >= 1 && t >= p.switch_iter;
      u_forward_iter(X, stage2, u_omega(p, t), Va, Vb, Vh, &s_fail);
      float2* dst = hist + (long long)(t - c0 + 1) * vn;
      u_step_project(X, p.gamma[t - 1], p.P[b], Vh, Vb, red);  // V^t into Vb
      for (int e = threadIdx.x; e < N; e += blockDim.x) dst[e] = Vb[e];
      float2* tmp = Va;
      Va = Vb;
      Vb = tmp;
      __syncthreads();
    }
    for (int t = c1; t > c0; --t) {
      const float2* hVa = hist + (long long)(t - c0) * vn;      // V^{t-1}
      const float2* hVb = hist + (long long)(t - c0 - 1) * vn;  // V^{t-2}
      for (int e = threadIdx.x; e < N; e += blockDim.x) {
        Va[e] = hVa[e];
        Vb[e] = hVb[e];
      }
      __syncthreads();
      u_adjoint_iter(p, X, L, smem, b, t, Va, Vb, Acc[0], Acc[1], Acc[2], &s_fail);
      float2* t0 = Acc[0];
      Acc[0] = Acc[1];
      Acc[1] = Acc[2];
      Acc[2] = t0;
    }
  }
  // Hbar for the channels as given: H_n = H / sigma_r
  float2* Hg = p.H_bar + (long long)b * X.m * X.Nt;
  for (int e = threadIdx.x; e < X.m * X.Nt; e += blockDim.x) {
    const int i = e / X.Nt;
    Hg[e] = cscale(Hb[e], rsqrtf(p.sigma2[(long long)b * X.K + i / X.Nr]));
  }
  if (threadIdx.x == 0 && s_fail != kOk) p.status[b] = s_fail;
}

}  // namespace
}  // namespace amm

struct amm_unrolled {
  int batch = 0, K = 0, Nt = 0, Nr = 0, d = 0, T = 0, ck = 0, nseg = 0, switch_iter = 0, extrapolate = 1;
  int smem = 0;
  cudaStream_t stream = nullptr;
  float2* ckpt = nullptr;
  float2* hist = nullptr;
  int* status = nullptr;
  const void* H = nullptr;
  const float *sigma2 = nullptr, *alpha = nullptr, *P = nullptr, *gamma = nullptr;
  bool forward_done = false;
  std::string err;
};

static thread_local std::string g_unrolled_err;

static amm_status u_fail(amm_unrolled* u, amm_status s, const std::string& msg) {
  if (u) u->err = msg;
  g_unrolled_err = msg;
  return s;
}

extern "C" amm_status amm_unrolled_create(amm_unrolled** out, int batch, const amm_dims* dims, int T, int ckpt_every,
                                          int switch_iter, int extrapolate, void* stream) {
  if (!out || !dims || batch < 1 || T < 1 || ckpt_every < 1)
    return u_fail(nullptr, AMM_EINVAL, "amm_unrolled_create: null pointer, batch < 1, T < 1 or ckpt_every < 1");
  *out = nullptr;
  const amm_dims& D = *dims;
  if (D.cells != 1) return u_fail(nullptr, AMM_EUNSUPPORTED, "amm_unrolled_create: one cell per instance only");
  if (D.users < 1 || D.nt < 1 || D.nr < 1 || D.nr > amm::kMaxNr || D.d < 1 || D.d > D.nr)
    return u_fail(nullptr, AMM_EINVAL, "amm_unrolled_create: dims out of range (1 <= d <= nr <= 4)");
  const amm::ULayout L = amm::u_layout(D.users, D.nt, D.nr, D.d);
  if (L.total > amm::kSmemMax - 1024)
    return u_fail(nullptr, AMM_EUNSUPPORTED, "amm_unrolled_create: instance too large for shared memory");
  amm_unrolled* u = new (std::nothrow) amm_unrolled();
  if (!u) return u_fail(nullptr, AMM_ENOMEM, "amm_unrolled_create: out of host memory");
  u->batch = batch;
  u->K = D.users;
  u->Nt = D.nt;
  u->Nr = D.nr;
  u->d = D.d;
  u->T = T;
  u->ck = ckpt_every;
  u->nseg = (T + ckpt_every - 1) / ckpt_every;
  u->switch_iter = switch_iter;
  u->extrapolate = extrapolate ? 1 : 0;
  u->smem = L.total;
  u->stream = static_cast<cudaStream_t>(stream);
  const long long vn = (long long)D.nt * D.users * D.d;
  cudaError_t e;
  if ((e = cudaMalloc(&u->ckpt, sizeof(float2) * vn * (2 * u->nseg + 1) * batch)) ||
      (e = cudaMalloc(&u->hist, sizeof(float2) * vn * (u->ck + 2) * batch)) ||
      (e = cudaMalloc(&u->status, sizeof(int) * batch)) ||
      (e = cudaFuncSetAttribute(amm::u_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total)) ||
      (e = cudaFuncSetAttribute(amm::u_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total))) {
    std::string msg = std::string("amm_unrolled_create: ") + cudaGetErrorString(e);
    cudaFree(u->ckpt);
    cudaFree(u->hist);
    cudaFree(u->status);
    delete u;
    return u_fail(nullptr, e == cudaErrorMemoryAllocation ? AMM_ENOMEM : AMM_ECUDA, msg);
  }
  *out = u;
  return AMM_OK;
}

static amm::UParams u_params(amm_unrolled* u) {
  amm::UParams p;
  memset(&p, 0, sizeof p);
  p.batch = u->batch;
  p.K = u->K;
  p.Nt = u->Nt;
  p.Nr = u->Nr;
  p.d = u->d;
  p.T = u->T;
  p.ck = u->ck;
  p.nseg = u->nseg;
  p.switch_iter = u->switch_iter;
  p.extrapolate = u->extrapolate;
  p.H = static_cast<const float2*>(u->H);
  p.sigma2 = u->sigma2;
  p.alpha = u->alpha;
  p.P = u->P;
  p.gamma = u->gamma;
  p.ckpt = u->ckpt;
  p.hist = u->hist;
  p.status = u->status;
  return p;
}

extern "C" amm_status amm_unrolled_forward(amm_unrolled* u, const void* H, const float* alpha, const float* sigma2,
                                           const float* P, const void* V0, const float* gamma, double* wsr) {
  if (!u) return AMM_EINVAL;
  if (!H || !alpha || !sigma2 || !P || !V0 || !gamma || !wsr)
    return u_fail(u, AMM_EINVAL, "amm_unrolled_forward: every pointer is required");
  u->H = H;
  u->alpha = alpha;
  u->sigma2 = sigma2;
  u->P = P;
  u->gamma = gamma;
  amm::UParams p = u_params(u);
  p.V0 = static_cast<const float2*>(V0);
  p.wsr = wsr;
  amm::u_forward_kernel<<<u->batch, amm::kUThreads, u->smem, u->stream>>>(p);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return u_fail(u, AMM_ECUDA, std::string("amm_unrolled_forward: ") + cudaGetErrorString(e));
  u->forward_done = true;
  return AMM_OK;
}

extern "C" amm_status amm_unrolled_backward(amm_unrolled* u, const double* wsr_bar, float* gamma_bar, void* H_bar) {
  if (!u) return AMM_EINVAL;
  if (!wsr_bar || !gamma_bar || !H_bar) return u_fail(u, AMM_EINVAL, "amm_unrolled_backward: every pointer is required");
  if (!u->forward_done) return u_fail(u, AMM_EINVAL, "amm_unrolled_backward before amm_unrolled_forward");
  amm::UParams p = u_params(u);
  p.wsr_bar = wsr_bar;
  p.gamma_bar = gamma_bar;
  p.H_bar = static_cast<float2*>(H_bar);
  amm::u_backward_kernel<<<u->batch, amm::kUThreads, u->smem, u->stream>>>(p);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return u_fail(u, AMM_ECUDA, std::string("amm_unrolled_backward: ") + cudaGetErrorString(e));
  return AMM_OK;
}

extern "C" amm_status amm_unrolled_status(amm_unrolled* u, int* status_dev) {
  if (!u || !status_dev) return AMM_EINVAL;
  const cudaError_t e =
      cudaMemcpyAsync(status_dev, u->status, sizeof(int) * u->batch, cudaMemcpyDeviceToDevice, u->stream);
  return e == cudaSuccess ? AMM_OK : u_fail(u, AMM_ECUDA, cudaGetErrorString(e));
}

extern "C" const char* amm_unrolled_last_error(amm_unrolled* u) {
  return u ? u->err.c_str() : g_unrolled_err.c_str();
}

extern "C" void amm_unrolled_destroy(amm_unrolled* u) {
  if (!u) return;
  cudaFree(u->ckpt);
  cudaFree(u->hist);
  cudaFree(u->status);
  delete u;
}
