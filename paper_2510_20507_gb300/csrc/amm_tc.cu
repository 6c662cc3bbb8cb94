// Fused A-MMMSE iteration kernel on the fifth-generation tensor cores
// (tcgen05, sm_103a): same algorithm and per-user FP64 solves as the plain
// kernel, but the two complex GEMMs of each iteration run as real BF16
// products with FP32 accumulation in tensor memory.
//
// Real embedding (one M = 128 tile per GEMM; single cell, 2m <= 128, 2Nt <= 128):
//   forward   [Zr; Zi] = [[Hr, -Hi], [Hi, Hr]] [Vr; Vi]            (A1 = H_real, B1 = V_real^T)
//   gradient  [Gr; Gi] = [[Hr^T, Hi^T], [-Hi^T, Hr^T]] [Yr; Yi]    (A2 = H_real^T, B2 = Y_real^T)
// so G = H^H Y exactly as the gradient of eq. (14).  BF16X3 splits every
// operand x = hi + lo and accumulates hi*hi + hi*lo + lo*hi.
//
// Tensor memory holds the FP32 state between iterations: Z(V^{t-1}) and
// Z(V^{t-2}) (two forward accumulators used alternately, so the
// extrapolated receiver input Z(Vhat) = (1+w) Z(V^{t-1}) - w Z(V^{t-2}) needs
// no extra GEMM), the gradient accumulator, and V^{t-1}, V^{t-2} in the same
// row layout as the gradient (lane p = row p of [Vr; Vi]), so the
// extrapolation, step and projection of eqs. (13), (15), (17) are lane-local.
#include <math.h>

#include "amm_device.cuh"
#include "amm_tc.cuh"

namespace amm {

// Number of bf16 terms each FP32 operand is split into: 1 (BF16), 2 (hi + lo,
// products hi*hi + hi*lo + lo*hi) or 3 (hi + mid + lo, products hi*hi +
// hi*mid + mid*hi + mid*mid + hi*lo + lo*hi, about FP32 accuracy).
__host__ __device__ inline int tc_splits(int prec) { return prec == 3 ? 3 : (prec == 2 ? 2 : 1); }
// With three terms the gradient GEMM reads H_real^T as the MN-major view of
// the forward operand instead of keeping a K-major copy: the same 8 x 16-byte
// core matrices, with 8-row groups of the forward operand now its K direction.
__host__ __device__ inline bool tc_mn_gradient(int prec) { return prec == 3; }

struct TcLayout {
  Layout base;  // the small per-user region (offsets from the plain plan)
  int K1p, K2p, Np, Bk, ncols, ns;
  bool mn;
  int off_A1[3], off_A2[3], off_B[3], off_Zs, off_L, off_Zo, end_ops;
  int total;
  bool ok;
};

__host__ __device__ inline TcLayout plan_tc(const InstDesc& D, int budget, int lanczos_steps, int prec) {
  TcLayout T;
  T.base = plan_layout(D, 0, lanczos_steps);  // budget 0: only the small region
  const int m = T.base.m, n = T.base.n;
  T.ns = tc_splits(prec);
  T.mn = tc_mn_gradient(prec);
  // the MN-major view spans all 128 rows of the gradient tile: keep K1 at 128
  T.K1p = T.mn ? 128 : align_up(2 * D.Nt, 16);
  T.K2p = align_up(2 * m, 16);
  T.Np = align_up(n < 16 ? 16 : n, 16);
  T.Bk = T.K1p > T.K2p ? T.K1p : T.K2p;
  int need = 5 * T.Np;
  T.ncols = 32;
  while (T.ncols < need) T.ncols <<= 1;
  int off = align_up(T.base.total, 1024);
  for (int s = 0; s < 3; ++s) {
    T.off_A1[s] = off;
    if (s < T.ns) off += 128 * T.K1p * 2;
  }
  for (int s = 0; s < 3; ++s) {
    T.off_A2[s] = off;
    if (s < T.ns && !T.mn) off += 128 * T.K2p * 2;
  }
  for (int s = 0; s < 3; ++s) {
    T.off_B[s] = off;
    if (s < T.ns) off += T.Np * T.Bk * 2;
  }
  T.end_ops = off;
  T.off_Zs = off;  off += m * T.base.ldz * 8;
  off = align_up(off, 16);
  const int szL = lanczos_elems(D) * 8;
  T.off_L = -1;
  if (off + szL <= budget) { T.off_L = off; off += szL; }
  // the users' own-stream blocks of Z, compact (lets the extrapolation
  // overwrite the Z staging buffer while the solves run)
  const int szZo = T.base.CK * D.Nr * D.d * 8;
  T.off_Zo = -1;
  if (off + szZo <= budget) { T.off_Zo = off; off += szZo; }
  T.total = off;
  T.ok = D.C == 1 && 2 * m <= 128 && 2 * D.Nt <= 128 && T.ncols <= 512 && off <= budget;
  return T;
}

// ||F_k||_2 by the general Lanczos form for shapes the row-blocked form
// does not take: with the FP32 channel copied into the idle Z staging
// buffer, or (when it does not fit there) summed from the bf16 split terms.
// Not inlined: they keep their registers out of the kernel's.
static __device__ __noinline__ float tc_lanczos_staged(const InstDesc& D, const Layout& Ly, const float2* Hg,
                                                       float2* Zs, int ldz, const float2* sU, const float2* sP,
                                                       const float* alpha_u, float2* QL, float2* ly, float2* lz,
                                                       float2* lD, float* ta, float* tb, double* red, float* bcast) {
  const int m = Ly.m, Nt = D.Nt;
  for (int e = threadIdx.x; e < m * Nt; e += blockDim.x) {
    const int i = e / Nt, q = e - i * Nt;
    Zs[(long long)i * ldz + q] = Hg[e];
  }
  __syncthreads();
  return lanczos_norm(
      D, Ly, [&](int i, int q) { return Zs[(long long)i * ldz + q]; }, sU, sP, alpha_u, QL, ly, lz, lD, ta, tb, red,
      bcast);
}
static __device__ __noinline__ float tc_lanczos_split(const InstDesc& D, const Layout& Ly, unsigned char* const* A1,
                                                      int NS, int K1p, const float2* sU, const float2* sP,
                                                      const float* alpha_u, float2* QL, float2* ly, float2* lz,
                                                      float2* lD, float* ta, float* tb, double* red, float* bcast) {
  const int m = Ly.m;
  return lanczos_norm(
      D, Ly,
      [&](int i, int q) {
        float re = 0.f, im = 0.f;
        for (int t = NS - 1; t >= 0; --t) {  // small terms first
          re += __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(A1[t] + tc::kmaj_off(i, q, K1p)));
          im += __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(A1[t] + tc::kmaj_off(m + i, q, K1p)));
        }
        return make_float2(re, im);
      },
      sU, sP, alpha_u, QL, ly, lz, lD, ta, tb, red, bcast);
}

template <class SolveT>
__global__ void __launch_bounds__(kThreads, 1) tc_iterate_kernel(IterParams p, int prec) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t mbar;
  __shared__ unsigned s_tmem;
  __shared__ int s_fail;
  __shared__ int s_ctrl[8];
  __shared__ float s_bcast;
  __shared__ ff s_rhoprev;  // R^{t-1} in float-float (hi NaN: none yet)

  const int b = p.order ? p.order[blockIdx.x] : (int)blockIdx.x;
  const InstDesc D = p.desc[b];
  Scalars* scg = p.sc + b;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int Nt = D.Nt;
  const TcLayout T = plan_tc(D, p.smem_budget, p.lanczos_steps, prec);
  const Layout& Ly = T.base;
  const int m = Ly.m, n = Ly.n, ldz = Ly.ldz;
  const int NS = T.ns;

  if (tid == 0) {
    const int st = scg->status;
    s_fail = (st == kNumeric || st == kTimeout) ? st : kOk;
    s_ctrl[0] = scg->t;
    s_ctrl[1] = scg->stage;
    s_ctrl[2] = scg->stage_iter;
    s_ctrl[3] = scg->last_stage;
    s_ctrl[4] = 0;
    s_ctrl[5] = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::su32(&mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (s_fail != kOk) return;  // before any tensor-memory allocation
  if (warp == 0) tc::tmem_alloc(&s_tmem, (unsigned)T.ncols);

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
  unsigned char* A1[3] = {smem + T.off_A1[0], smem + T.off_A1[1], smem + T.off_A1[2]};
  unsigned char* A2[3] = {smem + T.off_A2[0], smem + T.off_A2[1], smem + T.off_A2[2]};
  unsigned char* Bs[3] = {smem + T.off_B[0], smem + T.off_B[1], smem + T.off_B[2]};
  float2* Zs = reinterpret_cast<float2*>(smem + T.off_Zs);
  float2* QL = (T.off_L >= 0) ? reinterpret_cast<float2*>(smem + T.off_L) : p.Lws + D.l_off;
  float2* sZo = (T.off_Zo >= 0) ? reinterpret_cast<float2*>(smem + T.off_Zo) : nullptr;

  // per-instance scalars live in shared memory for the whole launch
  float* const s_alpha = reinterpret_cast<float*>(smem + Ly.off_alpha);
  const float* alpha_u = s_alpha;
  float* gamma_cg = p.gamma_c + D.c_off;
  for (int r = tid; r < Ly.CK; r += blockDim.x) s_alpha[r] = p.alpha[D.u_off + r];
  if (tid == 0) {
    cellf[48] = gamma_cg[0];
    s_rhoprev = ff_from_double(scg->rho_prev);
  }
  const float Pc = p.P[D.c_off];
  float* gamma_c = cellf + 48;
  float2* Vg = p.V + D.v_off;
  float2* Vpg = p.Vprev + D.v_off;
  const float2* Hg = p.H + D.h_off;

  // ---- zero the operand buffers (padding rows / K columns must read as 0)
  {
    uint4* z4 = reinterpret_cast<uint4*>(smem + T.off_A1[0]);
    const int n4 = (T.end_ops - T.off_A1[0]) / 16;
    for (int e = tid; e < n4; e += blockDim.x) z4[e] = make_uint4(0u, 0u, 0u, 0u);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const unsigned tbase = s_tmem;
  const int Np = T.Np;
  const unsigned colD1[2] = {0u, (unsigned)Np};
  const unsigned colD2 = 2u * Np;
  const unsigned colV[2] = {3u * Np, 4u * Np};

  // split x into NS bf16 terms
  auto split = [&](float x, __nv_bfloat16* t) {
    t[0] = __float2bfloat16_rn(x);
    float r = x - __bfloat162float(t[0]);
    if (NS > 1) {
      t[1] = __float2bfloat16_rn(r);
      r -= __bfloat162float(t[1]);
    }
    if (NS > 2) t[2] = __float2bfloat16_rn(r);
  };
  // split two values at once into NS packed bf16 pairs (word q holds term q
  // of x0 in its low half and of x1 in its high half); the paired
  // conversion rounds each half exactly as split() does
  auto split2 = [&](float x0, float x1, unsigned* w) {
    __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
    w[0] = reinterpret_cast<const unsigned&>(h);
    if (NS > 1) {
      x0 -= __low2float(h);
      x1 -= __high2float(h);
      h = __floats2bfloat162_rn(x0, x1);
      w[1] = reinterpret_cast<const unsigned&>(h);
    }
    if (NS > 2) {
      x0 -= __low2float(h);
      x1 -= __high2float(h);
      h = __floats2bfloat162_rn(x0, x1);
      w[2] = reinterpret_cast<const unsigned&>(h);
    }
  };
  auto put = [&](unsigned char* const* Ar, int row, int k, int Kp, const __nv_bfloat16* t, bool neg) {
    for (int q = 0; q < NS; ++q)
      *reinterpret_cast<__nv_bfloat16*>(Ar[q] + tc::kmaj_off(row, k, Kp)) = neg ? __hneg(t[q]) : t[q];
  };
  unsigned phase = 0;  // of mbar: the bulk copy below, then the MMA commits
  // ---- A operands from the normalised channel, staged into the idle Z
  //      buffer by the TMA bulk-copy engine (one row per copy) when its
  //      rows are wide enough
  const bool h_staged = Nt <= ldz;
  if (h_staged) stage_rows(Zs, ldz, Hg, Nt, m, Nt, &mbar, phase, p.spin_budget, &s_fail);
  for (int e = tid; e < m * Nt; e += blockDim.x) {
    const int i = e / Nt, q = e - i * Nt;
    const float2 h = h_staged ? Zs[(long long)i * ldz + q] : Hg[e];
    __nv_bfloat16 rt[3], it[3];
    split(h.x, rt);
    split(h.y, it);
    put(A1, i, q, T.K1p, rt, false);           // Hr
    put(A1, i, Nt + q, T.K1p, it, true);       // -Hi
    put(A1, m + i, q, T.K1p, it, false);       // Hi
    put(A1, m + i, Nt + q, T.K1p, rt, false);  // Hr
    if (!T.mn) {
      put(A2, q, i, T.K2p, rt, false);           // Hr^T
      put(A2, q, m + i, T.K2p, it, false);       // Hi^T
      put(A2, Nt + q, i, T.K2p, it, true);       // -Hi^T
      put(A2, Nt + q, m + i, T.K2p, rt, false);  // Hr^T
    }
  }

  // lane-owner mapping of the tensor-memory rows: warp w reads lanes of
  // quarter w%4 and the 16-column chunks h, h+2, ... (h = w/4)
  const int quarter = warp & 3, half = warp >> 2;
  const int R = quarter * 32 + lane;
  const unsigned lane_addr = tbase + ((unsigned)(quarter * 32) << 16);
  const int nchunks = Np / 16;

  // V state rows: R < Nt real part of row R, Nt <= R < 2Nt imaginary part
  auto load_state = [&](const float2* src, unsigned col) {
    for (int cc = half; cc < nchunks; cc += 2) {
      float v[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int c = cc * 16 + j;
        float x = 0.f;
        if (c < n && R < Nt) x = src[(long long)R * n + c].x;
        else if (c < n && R < 2 * Nt) x = src[(long long)(R - Nt) * n + c].y;
        v[j] = x;
      }
      tc::tmem_st16(lane_addr + col + cc * 16, v);
    }
    tc::tmem_wait_st();
  };
  // B1 = V_real^T, MN-major: for K index R (this lane's row of V_real), the
  // N entries c are contiguous in 16-byte rows of 8, so the lane stores each
  // 8-column piece of a split term with one 16-byte store.  Core matrices:
  // 8 K-rows x 16 B; stride 128 B along N, (Np/8) 128 B along K.
  auto put_B1 = [&](int cc, const float* v) {
    if (R >= T.K1p) return;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      unsigned t[4][3];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = cc * 16 + h * 8 + 2 * j;
        split2(c < n ? v[h * 8 + 2 * j] : 0.f, c + 1 < n ? v[h * 8 + 2 * j + 1] : 0.f, t[j]);
      }
      const int cb = cc * 2 + h;  // 8-column block
      const int off = (R >> 3) * (Np / 8) * 128 + cb * 128 + (R & 7) * 16;
      for (int q = 0; q < NS; ++q)
        *reinterpret_cast<uint4*>(Bs[q] + off) = make_uint4(t[0][q], t[1][q], t[2][q], t[3][q]);
    }
  };
  auto write_B1 = [&](unsigned col) {
    for (int cc = half; cc < nchunks; cc += 2) {
      float v[16];
      tc::tmem_ld16(lane_addr + col + cc * 16, v);
      put_B1(cc, v);
    }
  };
  // the products of the split terms: (a-term, b-term)
  const int npairs = (NS == 1) ? 1 : (NS == 2 ? 3 : 6);
  const int pa[6] = {0, 0, 1, 1, 0, 2}, pb[6] = {0, 1, 0, 1, 2, 0};
  // D = A * B over Kp; mn: A is the MN-major view of the forward operand (H_real^T)
  auto gemm = [&](unsigned dcol, unsigned char* const* Ar, int Kp, bool mn, bool bmn) -> bool {
    // operands written by the threads -> visible to the tensor core
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t idesc = tc::idesc_bf16(128, Np) | (mn ? (1u << 15) : 0u) | (bmn ? (1u << 16) : 0u);
      // no swizzle: LBO is the stride between core matrices along K, SBO along M/N,
      // for K-major and MN-major operands alike
      const unsigned kmaj_sbo = (unsigned)(Kp / 8) * 128u;
      const unsigned lbo_a = mn ? (unsigned)(T.K1p / 8) * 128u : 128u;
      const unsigned sbo_a = mn ? 128u : kmaj_sbo;
      const unsigned lbo_b = bmn ? (unsigned)(Np / 8) * 128u : 128u;
      const unsigned sbo_b = bmn ? 128u : kmaj_sbo;
      for (int kk = 0; kk < Kp / 16; ++kk) {
        const unsigned aoff = mn ? (unsigned)kk * 2u * lbo_a : (unsigned)kk * 256u;
        const unsigned boff = bmn ? (unsigned)kk * 2u * lbo_b : (unsigned)kk * 256u;
        for (int q = 0; q < npairs; ++q) {
          tc::mma_bf16(tbase + dcol, tc::smem_desc(tc::su32(Ar[pa[q]]) + aoff, lbo_a, sbo_a),
                       tc::smem_desc(tc::su32(Bs[pb[q]]) + boff, lbo_b, sbo_b), idesc, (kk > 0 || q > 0) ? 1u : 0u);
        }
      }
      tc::commit(&mbar);
    }
    const bool ok = tc::mbar_wait(&mbar, phase, p.spin_budget);
    phase ^= 1u;
    tc::fence_after_sync();
    if (!ok) {
      atomicExch(&s_fail, kTimeout);
      tc::mbar_wait(&mbar, phase ^ 1u, kDrainBudget);  // let the MMAs drain before the block moves on
    }
    __syncthreads();
    return s_fail == kOk;
  };

  int cur = 0, zc = 0;
  load_state(Vg, colV[0]);
  load_state(Vpg, colV[1]);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (p.extrapolate && s_ctrl[0] >= 3) {
    write_B1(colV[1]);
    gemm(colD1[1], A1, T.K1p, false, true);  // Z(V^{t-2})
  }
  write_B1(colV[0]);

  // the extrapolation can run beside the solves when the users fill warps 0-3
  // only (eight lanes per user in FP64, four in FP32) and the compact copy fits
  constexpr int kSolveLanes = std::is_same<SolveT, float>::value ? 4 : 8;
  const bool xo_ok = sZo != nullptr && kSolveLanes * Ly.CK <= 128 && blockDim.x == 256;
  ff rho = ff_from(0.f);
  for (int it = 0; it < p.n_iters && s_fail == kOk; ++it) {
    const int t = s_ctrl[0];
    const float omega = (p.extrapolate && t >= 3) ? (float)(t - 2) / (float)(t + 1) : 0.f;
    // ---- S2: Z = H V^{t-1} on the tensor cores
    if (!gemm(colD1[zc], A1, T.K1p, false, true)) break;
    // accumulator -> FP32 Z in shared memory (lane R < m: Re row R; m <= R < 2m: Im row R - m)
    for (int cc = half; cc < nchunks; cc += 2) {
      float v[16];
      tc::tmem_ld16(lane_addr + colD1[zc] + cc * 16, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int c = cc * 16 + j;
        if (c < n && R < m) Zs[(long long)R * ldz + c].x = v[j];
        else if (c < n && R < 2 * m) Zs[(long long)(R - m) * ldz + c].y = v[j];
      }
    }
    tc::fence_before_sync();
    __syncthreads();
    // ---- S3/S4: covariance, FP64 solves, rho = WSR(V^{t-1}), stage test.  When the
    //      extrapolation overlaps the solves, the users' own-stream blocks are copied
    //      out of Zs first (one cell: user r owns columns r d ..)
    const bool overlap = omega != 0.f && xo_ok;
    if (overlap)
      for (int e = tid; e < Ly.CK * D.Nr * D.d; e += blockDim.x) {
        const int row = e / D.d, q = e - row * D.d;
        sZo[e] = Zs[(long long)row * ldz + (row / D.Nr) * D.d + q];
      }
    covariance_phase(D, Ly, [&](int row, int c) { return Zs[(long long)row * ldz + c]; }, sQ);
    __syncthreads();
    // ---- S1 overlapped: while warps 0-3 solve, warps 4-7 (no users) form
    //      Z(Vhat) = (1+w) Z(V^{t-1}) - w Z(V^{t-2}) into Zs, all column chunks
    //      of their lane quarter; the solves read Z_own from the compact copy
    auto extrap_idle = [&]() {
      if (warp < 4) return;
      tc::fence_after_sync();
      for (int cc = 0; cc < nchunks; ++cc) {
        float v[16], vp[16];
        tc::tmem_ld16x2(lane_addr + colD1[zc] + cc * 16, lane_addr + colD1[zc ^ 1] + cc * 16, v, vp);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int c = cc * 16 + j;
          const float zh = (1.f + omega) * v[j] - omega * vp[j];
          if (c < n && R < m) Zs[(long long)R * ldz + c].x = zh;
          else if (c < n && R < 2 * m) Zs[(long long)(R - m) * ldz + c].y = zh;
        }
      }
      tc::fence_before_sync();
    };
    const bool want_rate = need_rate(s_ctrl[1], p.mode, it, p.n_iters);
    if (overlap)
      solve_phase<SolveT>(D, Ly, Zs, ldz, sQ, sU, sUW, sRho, alpha_u, true, want_rate, red, &s_fail, sZo,
                          extrap_idle);
    else
      solve_phase<SolveT>(D, Ly, Zs, ldz, sQ, sU, sUW, sRho, alpha_u, true, want_rate, red, &s_fail);
    if (s_fail != kOk) break;
    rho = want_rate ? rho_sum_ff(sRho, alpha_u, Ly.CK, red) : ff_from(0.f);
    if (tid == 0)
      stage_logic(s_ctrl, rho, s_rhoprev, p.mode, (float)p.eps1, (float)p.eps2, p.switch_iter, p.step_rule, p.tc);
    __syncthreads();
    if (s_ctrl[4]) break;
    const int stage = s_ctrl[1];
    const float2* sP = (stage == 2) ? sUW : sU;
    // ---- S1: Z(Vhat) = (1+w) Z(V^{t-1}) - w Z(V^{t-2}) into Zs (unless overlapped above)
    if (omega != 0.f && !overlap) {
      tc::fence_after_sync();
      for (int cc = half; cc < nchunks; cc += 2) {
        float v[16], vp[16];
        tc::tmem_ld16x2(lane_addr + colD1[zc] + cc * 16, lane_addr + colD1[zc ^ 1] + cc * 16, v, vp);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int c = cc * 16 + j;
          const float zh = (1.f + omega) * v[j] - omega * vp[j];
          if (c < n && R < m) Zs[(long long)R * ldz + c].x = zh;
          else if (c < n && R < 2 * m) Zs[(long long)(R - m) * ldz + c].y = zh;
        }
      }
      tc::fence_before_sync();
      __syncthreads();
    }
    // ---- S6: B2 = Y_real^T (K-major, K index: Re rows then Im rows)
    gradient_rhs_phase(
        D, Ly, [&](int row, int c) { return Zs[(long long)row * ldz + c]; }, sU, sP, alpha_u,
        [&](int r, int c, const float2* y) {
          const int Nr = D.Nr;
          if (Nr == 4) {
            // four consecutive K entries (rows r*4..r*4+3, then m + r*4..) share
            // one 8-byte piece of a core-matrix row: one store per split term
            unsigned r01[3], r23[3], i01[3], i23[3];
            split2(y[0].x, y[1].x, r01);
            split2(y[2].x, y[3].x, r23);
            split2(y[0].y, y[1].y, i01);
            split2(y[2].y, y[3].y, i23);
            for (int q = 0; q < NS; ++q) {
              *reinterpret_cast<uint2*>(Bs[q] + tc::kmaj_off(c, r * 4, T.K2p)) = make_uint2(r01[q], r23[q]);
              *reinterpret_cast<uint2*>(Bs[q] + tc::kmaj_off(c, m + r * 4, T.K2p)) = make_uint2(i01[q], i23[q]);
            }
          } else {
            for (int a = 0; a < Nr; ++a) {
              __nv_bfloat16 t[3];
              split(y[a].x, t);
              put(Bs, c, r * Nr + a, T.K2p, t, false);
              split(y[a].y, t);
              put(Bs, c, m + r * Nr + a, T.K2p, t, false);
            }
          }
        });
    for (int e = tid; e < n * (T.K2p - 2 * m); e += blockDim.x) {  // K padding of B2
      const int c = e / (T.K2p - 2 * m), k = 2 * m + e % (T.K2p - 2 * m);
      const __nv_bfloat16 z[3] = {__float2bfloat16_rn(0.f), __float2bfloat16_rn(0.f), __float2bfloat16_rn(0.f)};
      put(Bs, c, k, T.K2p, z, false);
    }
    __syncthreads();
    // ---- S5: step size, eq. (16).  The Z staging buffer is idle now (Y has been
    //      formed from it): when the FP32 channel fits there, Lanczos reads it
    //      from shared memory; otherwise it sums the bf16 split terms.
    {
      const int sflag = s_ctrl[6];
      float gk;
      if (sflag & 1) {
        float lam;
        if (lanczos_rows_ok(D, Ly, blockDim.x) && m * ldz >= (int)(blockDim.x >> 5) * 64) {
          // the channel straight from global memory into registers; the
          // staging buffer holds the warps' parts of Htilde^H z
          lam = lanczos_norm_rows(D, Ly, Hg, Nt, sU, sP, alpha_u, QL, lz, Zs, lD, ta, tb, red, &s_bcast);
        } else if (Nt <= ldz) {
          lam = tc_lanczos_staged(D, Ly, Hg, Zs, ldz, sU, sP, alpha_u, QL, ly, lz, lD, ta, tb, red, &s_bcast);
        } else {
          lam = tc_lanczos_split(D, Ly, A1, NS, T.K1p, sU, sP, alpha_u, QL, ly, lz, lD, ta, tb, red, &s_bcast);
        }
        gk = (lam > 0.f) ? 1.f / lam : 0.f;
        if ((sflag & 2) && tid == 0) gamma_c[0] = gk;
      } else {
        gk = (p.gamma_user > 0.f) ? p.gamma_user : gamma_c[0];
      }
      if (tid == 0) cellf[0] = gk;
    }
    // ---- S6/S7: G = H^H Y on the tensor cores
    if (!gemm(colD2, T.mn ? A1 : A2, T.K2p, T.mn, false)) break;
    const float gj = cellf[0];
    // Vtilde = Vhat - gamma G into the V^{t-2} slot and the block's ||Vtilde||^2
    // (four float-float partial sums: a chain of 8 additions, not 32)
    ff nacc[4] = {ff_from(0.f), ff_from(0.f), ff_from(0.f), ff_from(0.f)};
    for (int cc = half; cc < nchunks; cc += 2) {
      float g[16], v[16], vp[16];
      tc::tmem_ld16x3(lane_addr + colD2 + cc * 16, lane_addr + colV[cur] + cc * 16,
                      lane_addr + colV[cur ^ 1] + cc * 16, g, v, vp);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int c = cc * 16 + j;
        const float vh = (omega != 0.f) ? (1.f + omega) * v[j] - omega * vp[j] : v[j];
        float vt = vh - gj * g[j];
        if (!(c < n && R < 2 * Nt)) vt = 0.f;
        nacc[j & 3] = ff_add(nacc[j & 3], ff_from(vt * vt));
        v[j] = vt;
      }
      tc::tmem_st16(lane_addr + colV[cur ^ 1] + cc * 16, v);
    }
    const ff nrm = ff_add(ff_add(nacc[0], nacc[1]), ff_add(nacc[2], nacc[3]));
    tc::tmem_wait_st();
    // ||Vtilde||^2 in float-float, then the projection (eq. (15)) and
    // B1 = split(V^t) for the next forward GEMM
    const ff s = block_sum_ff(nrm, reinterpret_cast<float*>(red) + 80);
    const float scale = (s.hi > Pc) ? sqrtf(Pc / s.hi) : 1.f;
    for (int cc = half; cc < nchunks; cc += 2) {
      float v[16];
      tc::tmem_ld16(lane_addr + colV[cur ^ 1] + cc * 16, v);
      if (scale != 1.f) {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] *= scale;
        tc::tmem_st16(lane_addr + colV[cur ^ 1] + cc * 16, v);
      }
      put_B1(cc, v);
    }
    tc::tmem_wait_st();
    if (tid == 0) {
      s_rhoprev = rho;
      s_ctrl[3] = stage;
      s_ctrl[0] = t + 1;
      s_ctrl[5] += 1;
    }
    tc::fence_before_sync();
    __syncthreads();
    cur ^= 1;
    zc ^= 1;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  // ---- write the iterate back (lane R holds row R of [Vr; Vi])
  if (s_fail == kOk || s_fail == kNotConv) {
    for (int cc = half; cc < nchunks; cc += 2) {
      float v[16], vp[16];
      tc::tmem_ld16x2(lane_addr + colV[cur] + cc * 16, lane_addr + colV[cur ^ 1] + cc * 16, v, vp);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int c = cc * 16 + j;
        if (c < n && R < Nt) {
          Vg[(long long)R * n + c].x = v[j];
          Vpg[(long long)R * n + c].x = vp[j];
        } else if (c < n && R < 2 * Nt) {
          Vg[(long long)(R - Nt) * n + c].y = v[j];
          Vpg[(long long)(R - Nt) * n + c].y = vp[j];
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, (unsigned)T.ncols);
  if (tid == 0) {
    scg->t = s_ctrl[0];
    scg->rho_prev = ff_to_double(s_rhoprev);
    for (int k = 0; k < 1; ++k) gamma_cg[k] = gamma_c[k];
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

cudaError_t tc_set_smem(int bytes) {
  cudaError_t e = cudaFuncSetAttribute(tc_iterate_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_iterate_kernel<ff>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(tc_iterate_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}
// solves: 0 FP32, 1 FP64, 2 float-float
void tc_launch(int solves, int grid, int smem, cudaStream_t st, const IterParams& p, int prec) {
  if (solves == 1) tc_iterate_kernel<double><<<grid, kThreads, smem, st>>>(p, prec);
  else if (solves == 2) tc_iterate_kernel<ff><<<grid, kThreads, smem, st>>>(p, prec);
  else tc_iterate_kernel<float><<<grid, kThreads, smem, st>>>(p, prec);
}

// Host-side query: can every instance of the batch use the tensor-core
// kernel, and with how much shared memory?
int tc_plan_bytes(const InstDesc* desc, int batch, int budget, int lanczos_steps, int prec) {
  int mx = 0;
  for (int b = 0; b < batch; ++b) {
    const TcLayout T = plan_tc(desc[b], budget, lanczos_steps, prec);
    if (!T.ok) return -1;
    if (T.total > mx) mx = T.total;
  }
  return mx;
}

}  // namespace amm
