// NLINV pass kernels: batched row and column transforms over the coil planes with the pointwise steps of
// Eq. 2 and Eq. 3 fused into their loads and stores, CG vector updates, and deterministic FP64 reductions.
//
// Geometry.  A plane is N x N complex64, row-major, natural FFT order.  Omega (M_Omega of Eq. 2) is the square of
// indices e with e < f or e >= N - f in both axes (f = fov).  Image-domain intermediates only matter on Omega, so
// they are kept "compact": a T buffer holds J planes of N rows x Wc = 2f columns (the Omega columns), and the
// coil images c_j and the per-coil channel products hold J planes of Wc x Wc.  Compact index cc of natural
// index e: cc = e for e < f, cc = e - (N - 2f) for e >= N - f.
//
// Vectors of the unknown x = (rho, chat_1 .. chat_J) hold 1 + J planes: plane 0 is rho, planes 1..J chat_j.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "fft_core.cuh"

namespace nlv {

// ------------------------------------------------------------------------------------------ arguments ----
enum Reduce : int {
  RED_NONE = 0,       // the block partials are summed into Scalars::last
  RED_RESID = 1,      // Scalars::resid[slot] = sqrt(sum)       (|y - F x_n|)
  RED_RR_INIT = 2,    // Scalars::rr = sum                      (|b|^2 at the start of CG)
  RED_PQ = 3,         // Scalars::alpha = rr / sum              (sum = Re<p, A p>)
  RED_RR_UPDATE = 4,  // Scalars::beta = sum / rr, rr = sum     (|r_new|^2)
};

constexpr int kMaxNewton = 64;

// Scalars of the CG and Newton iterations, kept in device memory (FP64).
struct Scalars {
  double rr;                     // |r|^2 of the current CG residual
  double alpha;                  // CG step length
  double beta;                   // CG direction update
  double pq;                     // last Re<p, A p>
  double last;                   // result of a RED_NONE reduction
  double resid[kMaxNewton + 1];  // |y - F x_n| per Newton step
  int flags;                     // bit 0: CG breakdown (a non-finite |r|^2 or Re<p, A p>)
  unsigned ticket;               // completion counter of the last-block reduction
};

struct KArgs {
  int N, J, f, Wc;          // grid side, coils, half-width of Omega, compact width 2f
  int nrows;                // row passes: rows of the coil planes (J*N); column passes: J
  int coil_blocks;          // row passes with a rho part: blocks that work on coil rows
  const float* wtab;        // Sobolev weight w(k) = (1 + a |k|^2)^(-l/2), N x N natural order
  float alpha;              // alpha_n of Eq. 3 for the normal operator and the right-hand side
  int pupd;                 // CG passes: first form p = r + beta p (beta from Scalars) and write it back
  const float2* src;        // main input planes
  float2* dst;              // main output planes
  const float2* rho;        // rho of the linearisation point (natural N x N)
  const float2* drho;       // rho part of the direction (natural N x N)
  const float2* coil;       // c_j on Omega, compact J x Wc x Wc
  const float2* cimg;       // image-domain coils (natural J x N x N), forward simulation only
  float2* zsum;             // conj(c_j) z_j on Omega, compact J x Wc x Wc
  const uint8_t* mask;      // sampling pattern P, N x N
  const float2* y;          // data, J x N x N
  const float2* p;          // CG direction, (1+J) planes
  const float2* x;          // Newton iterate, (1+J) planes
  const float2* xref;       // regularisation centre, (1+J) planes
  float2* r;                // CG residual, (1+J) planes
  float2* pout;             // CG direction written by the right-hand side pass
  float2* dx;               // CG solution, (1+J) planes
  const float2* twA;        // twiddles of the split (N1, N2)
  const float2* twB;        // twiddles of the split (N2, N1)
  double* partials;         // one double per block
  Scalars* sc;
  int reduce;               // Reduce
  int slot;                 // RED_RESID index
};

// ------------------------------------------------------------------------------- dependent launches ----
// Every kernel is launched with programmatic stream serialisation: it may be scheduled while the kernel before it
// in the stream is still running.  griddepcontrol.wait blocks until that kernel has completed and its memory is
// visible, so it must come before the first global memory access; launch_dependents then lets the next kernel be
// scheduled as soon as every block of this one has started.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ------------------------------------------------------------------------------------------- geometry ----
__device__ __forceinline__ bool in_omega(int e, int N, int f) { return e < f || e >= N - f; }
__device__ __forceinline__ int to_compact(int e, int N, int f) { return e < f ? e : e - (N - 2 * f); }
__device__ __forceinline__ int to_natural(int cc, int N, int f) { return cc < f ? cc : cc + (N - 2 * f); }

// Sobolev weight of W (Sec. 3.1) at natural index (k1, k2), from the table built on the host in double precision.
__device__ __forceinline__ float sobolev_w(int k1, int k2, const KArgs& A) {
  return __ldg(&A.wtab[(size_t)k1 * A.N + k2]);
}

// beta of the pending direction update p = r + beta p (CG, Table 1)
__device__ __forceinline__ float cg_beta(const KArgs& A) { return (float)A.sc->beta; }

// ----------------------------------------------------------------------------------------- reductions ----
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum (fixed tree), result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (warp == 0) {
    s = lane < nw ? red[lane] : 0.0;
    s = warp_sum(s);
  }
  return s;
}

__device__ __forceinline__ void finalize_scalar(Scalars* sc, int reduce, int slot, double total) {
  switch (reduce) {
    case RED_RESID: sc->resid[slot] = sqrt(total); break;
    case RED_RR_INIT: sc->rr = total; sc->beta = 0.0; break;
    case RED_PQ: {
      // The system of Eq. 3 is positive definite, so Re<p, A p> <= 0 (or |r|^2 = 0) only occurs once CG has
      // reached the rounding floor: the step is then empty.  Non-finite values are a breakdown.
      double rr = sc->rr, a = 0.0;
      sc->pq = total;
      if (!isfinite(total) || !isfinite(rr)) sc->flags |= 1;
      else if (rr != 0.0 && total > 0.0) a = rr / total;
      sc->alpha = a;
      break;
    }
    case RED_RR_UPDATE: {
      double rr = sc->rr;
      sc->beta = (rr != 0.0) ? total / rr : 0.0;
      sc->rr = total;
      break;
    }
    default: sc->last = total; break;
  }
}

// Every thread passes its FP32 partial; per-block sums in FP64 go to partials[], and the last block to finish
// adds them in block order (so the result does not depend on scheduling) and updates the scalars.
__device__ __forceinline__ void grid_reduce(float mine, const KArgs& A) {
  __shared__ double red[32];
  __shared__ bool last;
  double s = block_sum((double)mine, red);
  if (threadIdx.x == 0) {
    A.partials[blockIdx.x] = s;
    __threadfence();
    unsigned t = atomicAdd(&A.sc->ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double acc = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) acc += __ldcg(&A.partials[i]);
  double total = block_sum(acc, red);
  if (threadIdx.x == 0) {
    finalize_scalar(A.sc, A.reduce, A.slot, total);
    A.sc->ticket = 0u;
  }
}

// ------------------------------------------------------------------------------------------ row passes ----
enum RowMode : int {
  ROW_W_IFFT = 0,        // T <- compact cols of FFT^-1_row(w * src / sqrt N)            (W^-1, first axis)
  ROW_PSF = 1,           // T <- compact cols of FFT^-1_row(P * FFT_row(T) / N)          (PSF step, Sec. 3.1)
  ROW_FFT_P_OUT = 2,     // dst <- P * FFT_row(T) / sqrt N                               (F, DF output)
  ROW_FFT_RESID = 3,     // dst <- y - P * FFT_row(T) / sqrt N, |dst|^2                  (Newton residual)
  ROW_P_IFFT = 4,        // T <- compact cols of FFT^-1_row(P * src / sqrt N)            (DF^H input)
  ROW_FFT_W_ADJ = 5,     // dst coil planes <- w FFT_row(T)/sqrt N; rho plane <- sum_j zsum_j (DF^H output)
  ROW_FFT_W_NORMAL = 6,  // as ADJ, plus alpha p; Re<p, q>                               (normal operator)
  ROW_FFT_W_RHS = 7,     // as ADJ, minus alpha (x - xref); r = p = b, dx = 0, |b|^2     (right-hand side)
  NUM_ROW_MODES = 8
};

template <int MODE> struct RowTraits {
  static constexpr bool load_compact = !(MODE == ROW_W_IFFT || MODE == ROW_P_IFFT);
  static constexpr bool inverse_first = (MODE == ROW_W_IFFT || MODE == ROW_P_IFFT);
  static constexpr bool has_rho = (MODE == ROW_FFT_W_ADJ || MODE == ROW_FFT_W_NORMAL || MODE == ROW_FFT_W_RHS);
  static constexpr bool reduces = (MODE == ROW_FFT_RESID || MODE == ROW_FFT_W_NORMAL || MODE == ROW_FFT_W_RHS);
};

template <int N1, int N2> struct RowCfg {
  using S = Split<N1, N2>;
  static constexpr int LANES = (256 / S::TL) >= 16 ? 16 : (256 / S::TL) >= 8 ? 8 : (256 / S::TL) >= 4 ? 4 : 2;
  static constexpr int THREADS = LANES * S::TL;
  static constexpr size_t SMEM = (size_t)LANES * S::SM_LANE * sizeof(float2);
};

// rho plane of the adjoint / normal / right-hand-side outputs: the sum of the channel products over the coils on
// Omega (the channel summation of Table 1) plus the mode's alpha term.  Each thread takes kRhoEPT consecutive
// pixels of one row; the coil loads are independent so that many are in flight at once.
constexpr int kRhoEPT = 8;

template <int MODE>
__device__ __forceinline__ float rho_part(const KArgs& A, int rb) {
  const int N = A.N, f = A.f, Wc = A.Wc, J = A.J;
  const long first = ((long)rb * blockDim.x + threadIdx.x) * kRhoEPT;
  float acc = 0.f;
  if (first >= (long)N * N) return acc;
  const int e1 = (int)(first / N), e20 = (int)(first % N);
  const bool row_in = in_omega(e1, N, f);
  const int cr = to_compact(e1, N, f);
  const float beta = (MODE == ROW_FFT_W_NORMAL && A.pupd) ? cg_beta(A) : 0.f;
#pragma unroll
  for (int t = 0; t < kRhoEPT; ++t) {
    const int e2 = e20 + t;
    const size_t o = (size_t)e1 * N + e2;
    float2 z = make_float2(0.f, 0.f);
    if (row_in && in_omega(e2, N, f)) {
      const float2* zp = A.zsum + (size_t)cr * Wc + to_compact(e2, N, f);
      const size_t stride = (size_t)Wc * Wc;
      int j = 0;
      for (; j + 4 <= J; j += 4) {
        float2 a0 = zp[(j + 0) * stride], a1 = zp[(j + 1) * stride];
        float2 a2 = zp[(j + 2) * stride], a3 = zp[(j + 3) * stride];
        z = cadd(z, cadd(cadd(a0, a1), cadd(a2, a3)));
      }
      for (; j < J; ++j) z = cadd(z, zp[j * stride]);
    }
    if constexpr (MODE == ROW_FFT_W_ADJ) {
      A.dst[o] = z;
    } else if constexpr (MODE == ROW_FFT_W_NORMAL) {
      float2 pv = A.p[o];
      if (A.pupd) {
        const float2 rv = A.r[o];
        pv = make_float2(fmaf(beta, pv.x, rv.x), fmaf(beta, pv.y, rv.y));
        const_cast<float2*>(A.p)[o] = pv;
      }
      float2 q = make_float2(fmaf(A.alpha, pv.x, z.x), fmaf(A.alpha, pv.y, z.y));
      A.dst[o] = q;
      acc += pv.x * q.x + pv.y * q.y;
    } else {
      float2 xv = A.x[o], xr = A.xref[o];
      float2 b = make_float2(z.x - A.alpha * (xv.x - xr.x), z.y - A.alpha * (xv.y - xr.y));
      A.r[o] = b;
      A.pout[o] = b;
      A.dx[o] = make_float2(0.f, 0.f);
      acc += b.x * b.x + b.y * b.y;
    }
  }
  return acc;
}

template <int N1, int N2, int MODE>
__global__ void __launch_bounds__(RowCfg<N1, N2>::THREADS) row_pass(const KArgs A) {
  using S = Split<N1, N2>;
  using T = RowTraits<MODE>;
  constexpr int N = S::N, TL = S::TL, E = S::E;
  extern __shared__ float2 smem[];
  pdl_enter();
  const int lane = threadIdx.x / TL, idx = threadIdx.x % TL;
  const int f = A.f, Wc = A.Wc;
  float acc = 0.f;

  if constexpr (T::has_rho) {
    if ((int)blockIdx.x >= A.coil_blocks) {
      acc = rho_part<MODE>(A, (int)blockIdx.x - A.coil_blocks);
      if constexpr (T::reduces) grid_reduce(acc, A);
      return;
    }
  }

  const int R = blockIdx.x * RowCfg<N1, N2>::LANES + lane;   // row of the stacked coil planes
  const bool active = R < A.nrows;
  const int e1 = R % N;
  float2* sm = smem + lane * S::SM_LANE;
  const float rs = rsqrtf((float)N);
  const float beta = (MODE == ROW_W_IFFT && A.pupd) ? cg_beta(A) : 0.f;
  float2 v[E];

  // ---- load, layout A: thread a < N1 holds row elements a + N1*m
  if (idx < N1) {
#pragma unroll
    for (int m = 0; m < N2; ++m) {
      const int e2 = idx + N1 * m;
      float2 val = make_float2(0.f, 0.f);
      if (active) {
        if constexpr (T::load_compact) {
          if (in_omega(e2, N, f)) val = A.src[(size_t)R * Wc + to_compact(e2, N, f)];
        } else if constexpr (MODE == ROW_W_IFFT) {
          const size_t o = (size_t)R * N + e2;
          float2 sv = A.src[o];
          if (A.pupd) {            // p = r + beta p on the coil planes, written back for the later passes
            const float2 rv = A.r[o];
            sv = make_float2(fmaf(beta, sv.x, rv.x), fmaf(beta, sv.y, rv.y));
            const_cast<float2*>(A.src)[o] = sv;
          }
          val = cscale(sv, sobolev_w(e1, e2, A) * rs);
        } else {  // ROW_P_IFFT
          val = A.mask[(size_t)e1 * N + e2] ? cscale(A.src[(size_t)R * N + e2], rs) : make_float2(0.f, 0.f);
        }
      }
      v[m] = val;
    }
  }

  if constexpr (T::inverse_first) {
    fft_AtoB<N1, N2, +1>(v, sm, A.twA, idx);
    // layout B: thread b < N2 holds elements b + N2*m; keep the Omega columns
    if (active && idx < N2) {
#pragma unroll
      for (int m = 0; m < N1; ++m) {
        const int e2 = idx + N2 * m;
        if (in_omega(e2, N, f)) A.dst[(size_t)R * Wc + to_compact(e2, N, f)] = v[m];
      }
    }
    return;
  } else {
    fft_AtoB<N1, N2, -1>(v, sm, A.twA, idx);
    if constexpr (MODE == ROW_PSF) {
      if (idx < N2) {
#pragma unroll
        for (int m = 0; m < N1; ++m) {
          const int e2 = idx + N2 * m;
          const float s = (active && A.mask[(size_t)e1 * N + e2]) ? rs * rs : 0.f;
          v[m] = cscale(v[m], s);
        }
      }
      fft_AtoB<N2, N1, +1>(v, sm, A.twB, idx);
      if (active && idx < N1) {
#pragma unroll
        for (int m = 0; m < N2; ++m) {
          const int e2 = idx + N1 * m;
          if (in_omega(e2, N, f)) A.dst[(size_t)R * Wc + to_compact(e2, N, f)] = v[m];
        }
      }
      return;
    } else {
      if (active && idx < N2) {
#pragma unroll
        for (int m = 0; m < N1; ++m) {
          const int e2 = idx + N2 * m;
          const size_t o = (size_t)R * N + e2;
          if constexpr (MODE == ROW_FFT_P_OUT) {
            A.dst[o] = A.mask[(size_t)e1 * N + e2] ? cscale(v[m], rs) : make_float2(0.f, 0.f);
          } else if constexpr (MODE == ROW_FFT_RESID) {
            float2 yv = A.y[o];
            float2 rv = A.mask[(size_t)e1 * N + e2] ? csub(yv, cscale(v[m], rs)) : yv;
            A.dst[o] = rv;
            acc += rv.x * rv.x + rv.y * rv.y;
          } else {
            const float2 val = cscale(v[m], sobolev_w(e1, e2, A) * rs);
            const size_t oc = (size_t)A.N * A.N + o;      // coil planes follow the rho plane
            if constexpr (MODE == ROW_FFT_W_ADJ) {
              A.dst[oc] = val;
            } else if constexpr (MODE == ROW_FFT_W_NORMAL) {
              float2 pv = A.p[oc];
              float2 q = make_float2(fmaf(A.alpha, pv.x, val.x), fmaf(A.alpha, pv.y, val.y));
              A.dst[oc] = q;
              acc += pv.x * q.x + pv.y * q.y;
            } else {  // ROW_FFT_W_RHS
              float2 xv = A.x[oc], xr = A.xref[oc];
              float2 b = make_float2(val.x - A.alpha * (xv.x - xr.x), val.y - A.alpha * (xv.y - xr.y));
              A.r[oc] = b;
              A.pout[oc] = b;
              A.dx[oc] = make_float2(0.f, 0.f);
              acc += b.x * b.x + b.y * b.y;
            }
          }
        }
      }
      if constexpr (T::reduces) grid_reduce(acc, A);
    }
  }
}

// --------------------------------------------------------------------------------------- column passes ----
enum ColMode : int {
  COL_IFFT_C = 0,         // coil <- Omega rows of FFT^-1_col(T) / sqrt N                 (W^-1, second axis)
  COL_PROD_FFT = 1,       // T <- FFT_col(M rho c_j) / sqrt N                             (F)
  COL_SIM_FFT = 2,        // T <- FFT_col(M rho cimg_j) / sqrt N                          (data simulation)
  COL_IFFT_PROD_FFT = 3,  // u = FFT^-1_col(T); T <- FFT_col(M (drho c_j + rho u))        (DF)
  COL_IFFT_ADJ_FFT = 4,   // z = M FFT^-1_col(T); zsum_j = conj(c_j) z; T <- FFT_col(conj(rho) z)   (DF^H)
  NUM_COL_MODES = 5
};

template <int N1, int N2> struct ColCfg {
  using S = Split<N1, N2>;
  static constexpr int C = 8;                       // adjacent compact columns per block
  static constexpr int THREADS = C * S::TL;
  static constexpr size_t SMEM = (size_t)C * S::SM_LANE * sizeof(float2);
};

template <int N1, int N2, int MODE>
__global__ void __launch_bounds__(ColCfg<N1, N2>::THREADS) col_pass(const KArgs A) {
  using S = Split<N1, N2>;
  constexpr int N = S::N, E = S::E, C = ColCfg<N1, N2>::C;
  extern __shared__ float2 smem[];
  pdl_enter();
  const int lane = threadIdx.x % C, idx = threadIdx.x / C;
  const int f = A.f, Wc = A.Wc;
  const int strips = (Wc + C - 1) / C;
  const int j = blockIdx.x / strips;
  const int cc = (blockIdx.x % strips) * C + lane;
  const bool active = cc < Wc && j < A.nrows;
  const int x2 = to_natural(cc, N, f);
  float2* sm = smem + lane * S::SM_LANE;
  const float rs = rsqrtf((float)N);
  const size_t tbase = (size_t)j * N * Wc + cc;       // T element (row e1) at tbase + e1*Wc
  const size_t cbase = (size_t)j * Wc * Wc + cc;      // compact coil element (row cr) at cbase + cr*Wc
  const float beta = (MODE == COL_IFFT_PROD_FFT && A.pupd) ? cg_beta(A) : 0.f;
  float2 v[E];

  if constexpr (MODE == COL_PROD_FFT || MODE == COL_SIM_FFT) {
    if (idx < N1) {
#pragma unroll
      for (int m = 0; m < N2; ++m) {
        const int e1 = idx + N1 * m;
        float2 val = make_float2(0.f, 0.f);
        if (active && in_omega(e1, N, f)) {
          float2 c = (MODE == COL_PROD_FFT) ? A.coil[cbase + (size_t)to_compact(e1, N, f) * Wc]
                                            : A.cimg[((size_t)j * N + e1) * N + x2];
          val = cmul(A.rho[(size_t)e1 * N + x2], c);
        }
        v[m] = val;
      }
    }
    fft_AtoB<N1, N2, -1>(v, sm, A.twA, idx);
    if (active && idx < N2) {
#pragma unroll
      for (int m = 0; m < N1; ++m) {
        const int e1 = idx + N2 * m;
        A.dst[tbase + (size_t)e1 * Wc] = cscale(v[m], rs);
      }
    }
    return;
  } else {
    if (idx < N1) {
#pragma unroll
      for (int m = 0; m < N2; ++m) {
        const int e1 = idx + N1 * m;
        v[m] = active ? A.src[tbase + (size_t)e1 * Wc] : make_float2(0.f, 0.f);
      }
    }
    fft_AtoB<N1, N2, +1>(v, sm, A.twA, idx);
    if constexpr (MODE == COL_IFFT_C) {
      if (active && idx < N2) {
#pragma unroll
        for (int m = 0; m < N1; ++m) {
          const int e1 = idx + N2 * m;
          if (in_omega(e1, N, f)) A.dst[cbase + (size_t)to_compact(e1, N, f) * Wc] = cscale(v[m], rs);
        }
      }
      return;
    } else {
      if (idx < N2) {
#pragma unroll
        for (int m = 0; m < N1; ++m) {
          const int e1 = idx + N2 * m;
          float2 out = make_float2(0.f, 0.f);
          if (active && in_omega(e1, N, f)) {
            const float2 u = cscale(v[m], rs);
            const size_t on = (size_t)e1 * N + x2;
            const float2 c = A.coil[cbase + (size_t)to_compact(e1, N, f) * Wc];
            const float2 rh = A.rho[on];
            if constexpr (MODE == COL_IFFT_PROD_FFT) {
              float2 dr = A.drho[on];
              if (A.pupd) {          // rho part of p = r + beta p (written later by the last row pass)
                const float2 rv = A.r[on];
                dr = make_float2(fmaf(beta, dr.x, rv.x), fmaf(beta, dr.y, rv.y));
              }
              out = cadd(cmul(dr, c), cmul(rh, u));
            } else {  // COL_IFFT_ADJ_FFT
              A.zsum[cbase + (size_t)to_compact(e1, N, f) * Wc] = cmulc(c, u);
              out = cmulc(rh, u);
            }
          }
          v[m] = out;
        }
      }
      fft_AtoB<N2, N1, -1>(v, sm, A.twB, idx);
      if (active && idx < N1) {
#pragma unroll
        for (int m = 0; m < N2; ++m) {
          const int e1 = idx + N1 * m;
          A.dst[tbase + (size_t)e1 * Wc] = cscale(v[m], rs);
        }
      }
    }
  }
}

// ------------------------------------------------------------------------------- per-size kernel table ----
struct SizeKernels {
  int N1, N2;
  int row_lanes, row_threads, col_lanes, col_threads;
  size_t row_smem, col_smem;
  const void* row[NUM_ROW_MODES];
  const void* col[NUM_COL_MODES];
};

template <int N1, int N2> SizeKernels make_size_kernels() {
  SizeKernels s{};
  s.N1 = N1;
  s.N2 = N2;
  s.row_lanes = RowCfg<N1, N2>::LANES;
  s.row_threads = RowCfg<N1, N2>::THREADS;
  s.row_smem = RowCfg<N1, N2>::SMEM;
  s.col_lanes = ColCfg<N1, N2>::C;
  s.col_threads = ColCfg<N1, N2>::THREADS;
  s.col_smem = ColCfg<N1, N2>::SMEM;
  s.row[ROW_W_IFFT] = (const void*)row_pass<N1, N2, ROW_W_IFFT>;
  s.row[ROW_PSF] = (const void*)row_pass<N1, N2, ROW_PSF>;
  s.row[ROW_FFT_P_OUT] = (const void*)row_pass<N1, N2, ROW_FFT_P_OUT>;
  s.row[ROW_FFT_RESID] = (const void*)row_pass<N1, N2, ROW_FFT_RESID>;
  s.row[ROW_P_IFFT] = (const void*)row_pass<N1, N2, ROW_P_IFFT>;
  s.row[ROW_FFT_W_ADJ] = (const void*)row_pass<N1, N2, ROW_FFT_W_ADJ>;
  s.row[ROW_FFT_W_NORMAL] = (const void*)row_pass<N1, N2, ROW_FFT_W_NORMAL>;
  s.row[ROW_FFT_W_RHS] = (const void*)row_pass<N1, N2, ROW_FFT_W_RHS>;
  s.col[COL_IFFT_C] = (const void*)col_pass<N1, N2, COL_IFFT_C>;
  s.col[COL_PROD_FFT] = (const void*)col_pass<N1, N2, COL_PROD_FFT>;
  s.col[COL_SIM_FFT] = (const void*)col_pass<N1, N2, COL_SIM_FFT>;
  s.col[COL_IFFT_PROD_FFT] = (const void*)col_pass<N1, N2, COL_IFFT_PROD_FFT>;
  s.col[COL_IFFT_ADJ_FFT] = (const void*)col_pass<N1, N2, COL_IFFT_ADJ_FFT>;
  return s;
}

}  // namespace nlv
