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
#include "tc_dft.cuh"

namespace nlv {

// ------------------------------------------------------------------------------------------ arguments ----
enum Reduce : int {
  RED_NONE = 0,       // the block partials are summed into Scalars::last
  RED_RESID = 1,      // Scalars::resid[slot] = sqrt(sum)       (|y - F x_n|)
  RED_RR_INIT = 2,    // Scalars::rr = sum                      (|b|^2 at the start of CG)
};

constexpr int kMaxNewton = 64;

// Scalars of the CG and Newton iterations, kept in device memory (FP64).
struct Scalars {
  double rr;                     // |r|^2 of the current CG residual (numerator of alpha)
  double rr0;                    // |b|^2 of the current CG solve (the reference of the rounding floor)
  double rr_prev;                // |r|^2 of the previous CG residual (denominator of the next beta)
  double alpha;                  // CG step length
  double beta;                   // CG direction update
  double pq;                     // last Re<p, A p>
  double last;                   // result of a RED_NONE reduction
  double resid[kMaxNewton + 1];  // |y - F x_n| per Newton step
  int cg_stop[kMaxNewton];       // per Newton step: the CG iteration that reached the rounding floor, -1 if none
  int flags;                     // bit 0: CG breakdown (a non-finite |r|^2 or Re<p, A p>);
                                 // bit 1: the current CG solve has reached the rounding floor (latched)
  unsigned ticket;               // completion counter of the last-block reduction
};

constexpr int kFlagBreakdown = 1;
constexpr int kFlagCgStopped = 2;
// Rounding floor of CG: the solve stops once |r|^2 <= kCgFloor2 |b|^2, i.e. |r| at the FP32 unit roundoff 2^-24
// relative to |b| (further iterations cannot improve a single-precision solution; left to run, the recursive
// residual decays into the FP32 denormal range, where the step lengths lose their precision).
constexpr double kCgFloor2 = 0x1p-48;

struct KArgs {
  int N, J, f, Wc;          // grid side, coils, half-width of Omega, compact width 2f
  int nrows;                // row passes: rows of the coil planes (J*N); column passes: J
  int rows_per_cta;         // row passes: consecutive coil rows handled by one block
  int rho_per_cta;          // row passes with a rho part: consecutive rho-plane pixels handled by one block
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
  int slot;                 // RED_RESID index; RED_RR_INIT and the CG step: the Newton step
  int iter;                 // CG step: index of the CG iteration
  const float2* q;          // CG step: A p
  long n2;                  // vector passes: number of float4 (two complex values each)
  // Re<p, A p> without a last-block tail: the normal-operator pass of the CG iteration only writes one FP64
  // partial per block into pq_part; the CG step, its one consumer, adds the n_pq partials itself to form alpha.
  double* pq_part;
  int n_pq;
  // |r|^2 likewise: the CG step writes one partial per block into rr_part, and the first pass of the next CG
  // iteration (its one consumer) adds the n_rr partials to form beta.  rr_part = NULL: beta from Scalars.
  double* rr_part;
  int n_rr;
  float coef;               // vector passes: second coefficient of out = alpha X + coef Y
  const void* tcB;          // tensor-core passes: the B tiles of the radix-16 DFT stage (tc_dft.cuh)
  int cgskip;               // a launch of the CG iteration: it returns at once when the solve has stopped
                            // (kCgSkipAfterWait, kCgSkipEarly: see cg_flags_early)
  int src_early;            // inputs written two or more launches back, read before the dependent-launch wait:
                            // the first CG pass's p (its first round's main loads), the CG step's r, dx and p
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

// True for a pass of the CG iteration whose solve has stopped at its rounding floor (Scalars::flags, latched by the
// CG step): the pass then skips its work -- the stopped solve's remaining iterations are empty steps (the dx they
// would leave is the one already there).  Only the CG step writes the flag, and every pass starts after the CG step
// before it has completed (dependent-launch wait), so all threads of a pass read the same value: each reads it
// itself, with no barrier.  (The CG step takes its own decision block-wide, inside cg_step_body.)
__device__ __forceinline__ bool cg_stopped(const KArgs& A) {
  return A.cgskip && (*(volatile const int*)&A.sc->flags & kFlagCgStopped) != 0;
}

// cgskip values.  kCgSkipEarly marks a pass whose flag may be read before its dependent-launch wait, so that the
// read overlaps the kernel before it instead of delaying this pass's first loads.  What a kernel may read before
// its wait: a kernel is scheduled only once every block of the kernel before it has passed its own wait (pdl_enter:
// wait, then launch_dependents), i.e. once the kernel two launches back has completed, so anything written two or
// more launches back (or before the stream reached the library's first kernel) is in place.  For the second to
// fifth passes of the CG iteration the flag's writer (the previous CG step) is two or more launches back; for the
// first pass it is the kernel just before.
constexpr int kCgSkipAfterWait = 1, kCgSkipEarly = 2;
__device__ __forceinline__ int cg_flags_early(const KArgs& A) {
  return A.cgskip == kCgSkipEarly ? *(volatile const int*)&A.sc->flags : 0;
}
// The stop test of a single-frame pass, given what cg_flags_early read before the wait.
__device__ __forceinline__ bool cg_stopped_after(const KArgs& A, int early_flags) {
  return A.cgskip == kCgSkipEarly ? (early_flags & kFlagCgStopped) != 0 : cg_stopped(A);
}

// ------------------------------------------------------------------------------------------- geometry ----
__device__ __forceinline__ bool in_omega(int e, int N, int f) { return e < f || e >= N - f; }
__device__ __forceinline__ int to_compact(int e, int N, int f) { return e < f ? e : e - (N - 2 * f); }
__device__ __forceinline__ int to_natural(int cc, int N, int f) { return cc < f ? cc : cc + (N - 2 * f); }

// beta of the pending direction update p = r + beta p (CG, Table 1)
__device__ __forceinline__ float cg_beta(const KArgs& A) { return (float)A.sc->beta; }

// ----------------------------------------------------------------------------------------- reductions ----
// Butterfly sum over the lanes of this warp that exist: lanes 0..cnt-1 (a block's last warp may be partial, and a
// row block can be narrower than a warp).  Only those lanes take part in the shuffles; a partner lane that does not
// exist counts as 0.  Valid in lane 0.
__device__ __forceinline__ double warp_sum(double v, int cnt = 32) {
  if (cnt >= 32) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
  }
  const unsigned mask = (1u << cnt) - 1u;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double w = __shfl_xor_sync(mask, v, o);
    if ((lane ^ o) < cnt) v += w;
  }
  return v;
}

// Lanes of the calling thread's warp that exist in this block.
__device__ __forceinline__ int warp_lanes() {
  const int rest = (int)blockDim.x - (int)(threadIdx.x & ~31u);
  return rest < 32 ? rest : 32;
}

// Deterministic block sum (fixed tree), result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v, warp_lanes());
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (warp == 0) {
    s = lane < nw ? red[lane] : 0.0;
    s = warp_sum(s, warp_lanes());
  }
  return s;
}

__device__ __forceinline__ void finalize_scalar(Scalars* sc, int reduce, int slot, double total) {
  switch (reduce) {
    case RED_RESID: sc->resid[slot] = sqrt(total); break;
    case RED_RR_INIT:           // a new CG solve starts: nothing has stopped yet
      sc->rr = total;
      sc->rr0 = total;
      sc->beta = 0.0;
      sc->flags &= ~kFlagCgStopped;
      sc->cg_stop[slot] = -1;
      break;
    default: sc->last = total; break;
  }
}

// Every thread passes its partial; per-block sums in FP64 go to partials[], and the last block to finish
// adds them in block order (so the result does not depend on scheduling) and updates the scalars.
// bid / nblk: this block's index and the number of blocks working on the same problem (the whole grid, or one
// frame's share of a batched grid).
__device__ __forceinline__ void grid_reduce(double mine, const KArgs& A, int bid, int nblk) {
  __shared__ double red[32];
  __shared__ bool last;
  double s = block_sum(mine, red);
  if (threadIdx.x == 0) {
    A.partials[bid] = s;
    __threadfence();
    unsigned t = atomicAdd(&A.sc->ticket, 1u);
    last = (t == (unsigned)nblk - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double acc = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) acc += __ldcg(&A.partials[i]);
  double total = block_sum(acc, red);
  if (threadIdx.x == 0) {
    finalize_scalar(A.sc, A.reduce, A.slot, total);
    A.sc->ticket = 0u;
  }
}

// ------------------------------------------------------------------------------------ async staging ----
// Side inputs of a pass (sampling pattern, weights, CG vectors, coil maps, rho) and the twiddle tables are copied
// into shared memory with cp.async at the start of every pass, together with the main loads, so that all load
// latencies overlap once instead of stalling the pointwise steps between the transforms.
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Copies nbytes (a multiple of 16, both addresses 16-byte aligned) with all threads of the block.
__device__ __forceinline__ void stage_bytes(void* sdst, const void* gsrc, int nbytes) {
  for (int i = threadIdx.x; i < nbytes / 16; i += blockDim.x)
    cp_async16((char*)sdst + 16 * i, (const char*)gsrc + 16 * i);
}

__host__ __device__ constexpr size_t align16(size_t v) { return (v + 15) / 16 * 16; }

// Rows R0 .. R0+nr-1 of rb bytes each (rb a multiple of 16) into consecutive rows of sdst: row R of gsrc, or row
// R mod N with `wrap` (tables of one plane shared by all coil planes); every run of consecutive source rows is one
// flat copy, so a thread issues about nr*rb / (16*blockDim.x) copies instead of one loop per row.
__device__ __forceinline__ void stage_rows(unsigned char* sdst, const void* gsrc, int R0, int nr, int rb, int N,
                                           bool wrap) {
  for (int l = 0; l < nr;) {
    const int R = R0 + l;
    const int e = wrap ? R % N : R;
    const int run = wrap ? min(nr - l, N - e) : nr - l;
    stage_bytes(sdst + (size_t)l * rb, (const unsigned char*)gsrc + (size_t)e * rb, run * rb);
    l += run;
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
  // side inputs staged per row: sampling-pattern row (bytes), weight row (floats), complex rows
  static constexpr bool s_mask = (MODE == ROW_PSF || MODE == ROW_FFT_P_OUT || MODE == ROW_FFT_RESID);
  static constexpr bool s_w = has_rho || MODE == ROW_W_IFFT;
};

// Shared-memory layout of a row pass (byte offsets), identical on host and device.
struct RowSmem {
  size_t xch, tw, mask, w, cplx, total;
};
__host__ __device__ inline RowSmem row_smem(int mode, int N, int lanes, int sm_lane) {
  RowSmem L{};
  const bool m = (mode == ROW_PSF || mode == ROW_FFT_P_OUT || mode == ROW_FFT_RESID);
  const bool w = (mode == ROW_FFT_W_ADJ || mode == ROW_FFT_W_NORMAL || mode == ROW_FFT_W_RHS || mode == ROW_W_IFFT);
  L.xch = 0;
  L.tw = align16((size_t)lanes * sm_lane * 8);
  L.mask = L.tw + align16((size_t)2 * N * 8);
  L.w = L.mask + (m ? align16((size_t)lanes * N) : 0);
  L.cplx = L.w + (w ? align16((size_t)lanes * N * 4) : 0);
  L.total = L.cplx + ((mode == ROW_FFT_RESID) ? (size_t)lanes * N * 8 : 0);
  return L;
}

#ifndef NLV_COL_C
#define NLV_COL_C 8
#endif

// Row passes run kRowCtasPerSM blocks per SM; a block holds up to kRowMaxThreads threads (whole lanes of TL
// threads) and loops over its share of rows when they do not fit at once.
constexpr int kRowMaxThreads = 320;
constexpr int kRowCtasPerSM = 2;

// rho plane of the adjoint / normal / right-hand-side outputs: the sum of the channel products over the coils on
// Omega (the channel summation of Table 1) plus the mode's alpha term.  Every block takes an equal slice of the
// plane after its rows, all of its threads working on it.  A thread takes two pixels per step (o and
// o + blockDim.x) and issues every load of both before the first use; the coil sum of a pixel runs over even and
// odd coils in two partial sums added at the end.
// Dot-product partials: a thread sums at most 32 products in FP32 (one row round, or two pixels of the rho slice)
// before adding them to its FP64 partial, so the FP32 summation length is bounded whatever the problem size.
template <int N, int MODE, bool STDF>
__device__ __forceinline__ double rho_slice(const KArgs& A, int bid) {
  // pixel and channel-product offsets in 32 bits: a plane has at most 1024^2 pixels, the J channel-product planes
  // at most 64 x 512^2 entries
  const int f = STDF ? N / 4 : A.f, Wc = STDF ? N / 2 : A.Wc, J = A.J;
  constexpr int plane = N * N;
  const int e_begin = bid * A.rho_per_cta;
  const int e_end = min(e_begin + A.rho_per_cta, plane);
  const float beta = (MODE == ROW_FFT_W_NORMAL && A.pupd) ? cg_beta(A) : 0.f;
  const int stride = Wc * Wc;
  const int bd = blockDim.x;
  double accd = 0.0;
  for (int o0 = e_begin + threadIdx.x; o0 < e_end; o0 += 2 * bd) {
    float acc = 0.f;
    float2 a[2], b[2];
    int zo[2];
    bool ok[2], om[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int o = o0 + k * bd;
      const int e1 = o / N, e2 = o - e1 * N;
      ok[k] = o < e_end;
      om[k] = ok[k] && in_omega(e1, N, f) && in_omega(e2, N, f);
      zo[k] = om[k] ? to_compact(e1, N, f) * Wc + to_compact(e2, N, f) : 0;
      a[k] = b[k] = make_float2(0.f, 0.f);
      if (ok[k]) {
        if constexpr (MODE == ROW_FFT_W_NORMAL) {
          a[k] = A.p[o];
          if (A.pupd) b[k] = A.r[o];
        } else if constexpr (MODE == ROW_FFT_W_RHS) {
          a[k] = A.x[o];
          b[k] = A.xref[o];
        }
      }
    }
    const float2 zero = make_float2(0.f, 0.f);
    float2 z00 = zero, z01 = zero, z10 = zero, z11 = zero;
    int j = 0;
    for (; j + 2 <= J; j += 2) {
      if (om[0]) { z00 = cadd(z00, A.zsum[zo[0]]); z01 = cadd(z01, A.zsum[zo[0] + stride]); }
      if (om[1]) { z10 = cadd(z10, A.zsum[zo[1]]); z11 = cadd(z11, A.zsum[zo[1] + stride]); }
      zo[0] += 2 * stride;
      zo[1] += 2 * stride;
    }
    if (j < J) {
      if (om[0]) z00 = cadd(z00, A.zsum[zo[0]]);
      if (om[1]) z10 = cadd(z10, A.zsum[zo[1]]);
    }
    const float2 z[2] = {cadd(z00, z01), cadd(z10, z11)};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (!ok[k]) continue;
      const int o = o0 + k * bd;
      if constexpr (MODE == ROW_FFT_W_ADJ) {
        A.dst[o] = z[k];
      } else if constexpr (MODE == ROW_FFT_W_NORMAL) {
        float2 pv = a[k];
        if (A.pupd) {
          pv = make_float2(fmaf(beta, pv.x, b[k].x), fmaf(beta, pv.y, b[k].y));
          const_cast<float2*>(A.p)[o] = pv;
        }
        const float2 q = make_float2(fmaf(A.alpha, pv.x, z[k].x), fmaf(A.alpha, pv.y, z[k].y));
        A.dst[o] = q;
        acc += pv.x * q.x + pv.y * q.y;
      } else {
        const float2 bb = make_float2(z[k].x - A.alpha * (a[k].x - b[k].x), z[k].y - A.alpha * (a[k].y - b[k].y));
        A.r[o] = bb;
        A.pout[o] = bb;
        A.dx[o] = make_float2(0.f, 0.f);
        acc += bb.x * bb.x + bb.y * bb.y;
      }
    }
    accd += (double)acc;
  }
  return accd;
}

// Side rows of the round starting at row R0 (sampling pattern, weights, data).  Every launch sequence writes these,
// if at all, two or more launches before the pass that stages them (the data rows of the gradient's second
// residual are the first residual, three launches back), never in the launch just before, so that a single-frame
// pass may stage them before its dependent-launch wait (see cg_flags_early for why that suffices).
template <int N, int MODE>
__device__ __forceinline__ void row_stage_side(const KArgs& A, const RowSmem& L, int R0, int r_end, int LANES,
                                               unsigned char* smem_raw) {
  using T = RowTraits<MODE>;
  const int nr = min(LANES, r_end - R0);
  if constexpr (T::s_mask) stage_rows(smem_raw + L.mask, A.mask, R0, nr, N, N, true);
  if constexpr (T::s_w) stage_rows(smem_raw + L.w, A.wtab, R0, nr, N * 4, N, true);
  if constexpr (MODE == ROW_FFT_RESID) stage_rows(smem_raw + L.cplx, A.y, R0, nr, N * 8, N, false);
}

// The twiddles and the first round's side rows of a single-frame row pass, issued before its dependent-launch
// wait (row_pass_body with PRE then skips them).
template <int N1, int N2, int MODE>
__device__ __forceinline__ void row_pass_prestage(const KArgs& A, int bid, unsigned char* smem_raw) {
  using S = Split<N1, N2>;
  constexpr int N = S::N;
  const int LANES = blockDim.x / S::TL;
  const RowSmem L = row_smem(MODE, N, LANES, S::SM_LANE);
  const int r_begin = bid * A.rows_per_cta;
  const int r_end = min(r_begin + A.rows_per_cta, A.nrows);
  stage_bytes(smem_raw + L.tw, A.twA, N * 8);
  stage_bytes(smem_raw + L.tw + N * 8, A.twB, N * 8);
  if (r_begin < r_end) row_stage_side<N, MODE>(A, L, r_begin, r_end, LANES, smem_raw);
}

// Row pass: block b takes the coil rows [b*rows_per_cta, (b+1)*rows_per_cta) of the stacked J*N rows, one lane
// (TL threads) per row, in as many rounds as its lanes need; passes with a rho part then take a slice of the rho
// plane.  All threads of the block run every round (inactive lanes carry zeros) because of the barriers.
// PRE: the twiddles and the first round's side rows were staged by row_pass_prestage, and the body itself waits for
// the kernel before (pdl_enter) and applies the stop test: before its first loads, or, for the first CG pass with
// src_early, right after the first round's main loads are issued.
template <int N1, int N2, int MODE, bool STDF = false, class TC = NoTc, bool PRE = false>
__device__ __forceinline__ void row_pass_body(const KArgs& A, int bid, int nblk, unsigned char* smem_raw,
                                              TC* tc = nullptr, int early_flags = 0) {
  using S = Split<N1, N2>;
  using T = RowTraits<MODE>;
  constexpr int N = S::N, TL = S::TL, E = S::E;
  static_assert(N2 == TL, "row passes assume N1 <= N2");
  const int LANES = blockDim.x / TL;
  // Two thread maps onto the rows of a round: layout A (N1 threads per row) packs the rows densely so that the
  // spare warps skip the layout-A steps; layout B uses N2 = TL threads per row (every thread).
  const int laneA = threadIdx.x / N1, idxA = threadIdx.x % N1;
  const bool mapA = (int)threadIdx.x < LANES * N1;
  const int laneB = threadIdx.x / N2, idxB = threadIdx.x % N2;
  const bool mapB = (int)threadIdx.x < LANES * N2;           // threads beyond the whole lanes stay idle
  const int f = STDF ? N / 4 : A.f, Wc = STDF ? N / 2 : A.Wc;
  float acc = 0.f;        // this round's products (at most N1 <= 16 complex values per thread)
  double accd = 0.0;      // FP64 sum of the rounds
  const RowSmem L = row_smem(MODE, N, LANES, S::SM_LANE);
  float2* smA = (float2*)(smem_raw + L.xch) + laneA * S::SM_LANE;
  float2* smB = (float2*)(smem_raw + L.xch) + laneB * S::SM_LANE;
  const float2* twA = (const float2*)(smem_raw + L.tw);
  const float2* twB = twA + N;
  const float rs = rsqrtf((float)N);
  const int r_begin = bid * A.rows_per_cta;
  const int r_end = min(r_begin + A.rows_per_cta, A.nrows);
  if (!PRE) {
    stage_bytes(smem_raw + L.tw, A.twA, N * 8);
    stage_bytes(smem_raw + L.tw + N * 8, A.twB, N * 8);
  }
  __shared__ float s_beta;       // beta of the direction update p = r + beta p (ROW_W_IFFT with pupd)
  bool waited = !PRE;
  // the dependent-launch wait and the stop test (the same for every thread of the block); true: leave the pass
  auto enter = [&]() -> bool {
    pdl_enter();
    waited = true;
    if (cg_stopped_after(A, early_flags)) {
      cp_async_wait_all();
      return true;
    }
    return false;
  };
  // with src_early the first CG pass issues its main loads (p) before the wait; every other pass waits first
  const bool early_main = PRE && MODE == ROW_W_IFFT && A.src_early;
  if (PRE && !early_main && enter()) return;

  for (int R0 = r_begin; R0 < r_end; R0 += LANES) {
  const int RA = R0 + laneA, RB = R0 + laneB;               // rows of the stacked coil planes in the two maps
  const bool activeA = mapA && RA < r_end, activeB = mapB && RB < r_end;
  const int e1A = RA % N;
  float2 v[E];

  // ---- direction update: the rows of r go to the exchange buffer (natural order, pitch N) while p is loaded
  if constexpr (MODE == ROW_W_IFFT) {
    if (A.pupd && waited) stage_rows(smem_raw + L.xch, A.r, R0, min(LANES, r_end - R0), N * 8, N, false);
  }

  // ---- main loads, layout A: thread a < N1 holds row elements a + N1*m (no stores until all are issued)
  if (mapA) {
#pragma unroll
    for (int m = 0; m < N2; ++m) {
      const int e2 = idxA + N1 * m;
      float2 val = make_float2(0.f, 0.f);
      if (activeA) {
        if constexpr (T::load_compact) {
          if (in_omega(e2, N, f)) val = A.src[(size_t)RA * Wc + to_compact(e2, N, f)];
        } else if constexpr (MODE == ROW_W_IFFT) {
          val = __ldcg(A.src + (size_t)RA * N + e2);     // from L2 (issued before the wait with src_early)
        } else {  // ROW_P_IFFT
          const float2 sv = A.src[(size_t)RA * N + e2];
          val = A.mask[(size_t)e1A * N + e2] ? sv : make_float2(0.f, 0.f);
        }
      }
      v[m] = val;
    }
  }
  if (!waited) {                 // src_early: the main loads are in flight; now the inputs of the kernel before
    if (enter()) return;
    if constexpr (MODE == ROW_W_IFFT) {
      if (A.pupd) stage_rows(smem_raw + L.xch, A.r, R0, min(LANES, r_end - R0), N * 8, N, false);
    }
  }

  // ---- staged side inputs (the twiddles were issued before the first round)
  if (!PRE || R0 != r_begin) row_stage_side<N, MODE>(A, L, R0, r_end, LANES, smem_raw);
  // beta from the |r|^2 partials of the CG step before, while the loads above are in flight (same order in every
  // block; block 0 publishes |r|^2 and beta for the CG step and the later passes of this iteration)
  if constexpr (MODE == ROW_W_IFFT) {
    if (A.pupd && R0 == r_begin) {
      if (A.rr_part) {
        __shared__ double red[32];
        double t = 0.0;
        for (int k = threadIdx.x; k < A.n_rr; k += blockDim.x) t += A.rr_part[k];
        t = block_sum(t, red);
        if (threadIdx.x == 0) {
          const double rp = A.sc->rr_prev;
          const double b = (rp != 0.0) ? t / rp : 0.0;
          s_beta = (float)b;
          if (bid == 0) { A.sc->rr = t; A.sc->beta = b; }
        }
      } else if (threadIdx.x == 0) {
        s_beta = cg_beta(A);
      }
    }
  }
  cp_async_wait_all();
  __syncthreads();

  if constexpr (MODE == ROW_W_IFFT) {
    // p = r + beta p (r from the exchange buffer) written back, then weight
    const float* sw = (const float*)(smem_raw + L.w) + (size_t)laneA * N;
    const float2* sr = (const float2*)(smem_raw + L.xch) + (size_t)laneA * N;
    if (activeA) {
#pragma unroll
      for (int m = 0; m < N2; ++m) {
        if (A.pupd) {
          const float2 rv = sr[idxA + N1 * m];
          v[m] = make_float2(fmaf(s_beta, v[m].x, rv.x), fmaf(s_beta, v[m].y, rv.y));
          const_cast<float2*>(A.src)[(size_t)RA * N + idxA + N1 * m] = v[m];
        }
        v[m] = cscale(v[m], sw[idxA + N1 * m] * rs);
      }
    }
    if (A.pupd) __syncthreads();   // the exchange below overwrites the staged rows of r
  } else if constexpr (MODE == ROW_P_IFFT) {
    if (mapA) {
#pragma unroll
      for (int m = 0; m < N2; ++m) v[m] = cscale(v[m], rs);
    }
  }

  if constexpr (T::inverse_first) {
    fft_AtoB2<N1, N2, +1, E, TC, false>(v, smA, idxA, mapA, smB, idxB, mapB, twA, tc);
    // layout B: thread b < N2 holds elements b + N2*m; keep the Omega columns
    if (activeB) {
#pragma unroll
      for (int m = 0; m < N1; ++m) {
        const int e2 = idxB + N2 * m;
        if (in_omega(e2, N, f)) A.dst[(size_t)RB * Wc + to_compact(e2, N, f)] = v[m];
      }
    }
  } else {
    // single-frame normal-operator pass: its rows of p (layout B) are loaded before the transform, so that their
    // latency overlaps it (the batched pass, HBM-bound, loads them after it: the early loads cost it 2.5 %)
    constexpr bool kEarlyP = MODE == ROW_FFT_W_NORMAL && PRE;
    float2 pB[kEarlyP ? N1 : 1];
    if constexpr (kEarlyP) {
      if (activeB) {
#pragma unroll
        for (int m = 0; m < N1; ++m) pB[m] = A.p[(size_t)N * N + (size_t)RB * N + idxB + N2 * m];
      }
    }
    // the PSF pass exchanges again right after: keep the closing barrier there
    fft_AtoB2<N1, N2, -1, E, TC, MODE == ROW_PSF>(v, smA, idxA, mapA, smB, idxB, mapB, twA, tc);
    const unsigned char* smask = smem_raw + L.mask + (size_t)laneB * N;
    if constexpr (MODE == ROW_PSF) {
      {
#pragma unroll
        for (int m = 0; m < N1; ++m) {
          const float sc = (activeB && smask[idxB + N2 * m]) ? rs * rs : 0.f;
          v[m] = cscale(v[m], sc);
        }
      }
      fft_AtoB2<N2, N1, +1, E, TC, false>(v, smB, idxB, mapB, smA, idxA, mapA, twB, tc);
      if (activeA) {
#pragma unroll
        for (int m = 0; m < N2; ++m) {
          const int e2 = idxA + N1 * m;
          if (in_omega(e2, N, f)) A.dst[(size_t)RA * Wc + to_compact(e2, N, f)] = v[m];
        }
      }
    } else {
      const float* sw = (const float*)(smem_raw + L.w) + (size_t)laneB * N;
      // staged rows of y; p, or x and x_ref, loaded into registers before any store
      const float2* scp = (const float2*)(smem_raw + L.cplx) + (size_t)laneB * N;
      constexpr int NV = (MODE == ROW_FFT_W_RHS) ? 2 : (MODE == ROW_FFT_W_NORMAL) ? 1 : 0;
      float2 a0[NV ? N1 : 1], a1[NV == 2 ? N1 : 1];
      if (NV && activeB) {
#pragma unroll
        for (int m = 0; m < N1; ++m) {
          const size_t oc = (size_t)N * N + (size_t)RB * N + idxB + N2 * m;
          if constexpr (MODE == ROW_FFT_W_NORMAL) {
            if constexpr (kEarlyP) a0[m] = pB[m];
            else a0[m] = A.p[oc];
          }
          if constexpr (MODE == ROW_FFT_W_RHS) {
            a0[m] = A.x[oc];
            a1[m] = A.xref[oc];
          }
        }
      }
      if (activeB) {
#pragma unroll
        for (int m = 0; m < N1; ++m) {
          const int e2 = idxB + N2 * m;
          const size_t o = (size_t)RB * N + e2;
          if constexpr (MODE == ROW_FFT_P_OUT) {
            A.dst[o] = smask[e2] ? cscale(v[m], rs) : make_float2(0.f, 0.f);
          } else if constexpr (MODE == ROW_FFT_RESID) {
            const float2 yv = scp[e2];
            const float2 rv = smask[e2] ? csub(yv, cscale(v[m], rs)) : yv;
            A.dst[o] = rv;
            acc += rv.x * rv.x + rv.y * rv.y;
          } else {
            const float2 val = cscale(v[m], sw[e2] * rs);
            const size_t oc = (size_t)N * N + o;      // coil planes follow the rho plane
            if constexpr (MODE == ROW_FFT_W_ADJ) {
              A.dst[oc] = val;
            } else if constexpr (MODE == ROW_FFT_W_NORMAL) {
              const float2 pv = a0[m];
              const float2 q = make_float2(fmaf(A.alpha, pv.x, val.x), fmaf(A.alpha, pv.y, val.y));
              A.dst[oc] = q;
              acc += pv.x * q.x + pv.y * q.y;
            } else {  // ROW_FFT_W_RHS
              const float2 xv = a0[m], xr = a1[m];
              const float2 b = make_float2(val.x - A.alpha * (xv.x - xr.x), val.y - A.alpha * (xv.y - xr.y));
              A.r[oc] = b;
              A.pout[oc] = b;
              A.dx[oc] = make_float2(0.f, 0.f);
              acc += b.x * b.x + b.y * b.y;
            }
          }
        }
      }
    }
  }
  if (R0 + LANES < r_end) __syncthreads();   // the next round restages the side rows and reuses the exchange
  if constexpr (T::reduces) {
    accd += (double)acc;
    acc = 0.f;
  }
  }  // rounds

  if constexpr (T::has_rho) accd += rho_slice<N, MODE, STDF>(A, bid);
  if constexpr (T::reduces) {
    if (MODE == ROW_FFT_W_NORMAL && A.pq_part) {
      __shared__ double red[32];
      const double sblk = block_sum(accd, red);
      if (threadIdx.x == 0) A.pq_part[bid] = sblk;
    } else {
      grid_reduce(accd, A, bid, nblk);
    }
  }
}

template <int N1, int N2, int MODE, bool STDF = false>
__global__ void __launch_bounds__(kRowMaxThreads, kRowCtasPerSM) row_pass(const KArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int early = cg_flags_early(A);
  row_pass_prestage<N1, N2, MODE>(A, blockIdx.x, smem_raw);
  row_pass_body<N1, N2, MODE, STDF, NoTc, true>(A, blockIdx.x, gridDim.x, smem_raw, nullptr, early);
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

// Shared-memory layout of a column pass (byte offsets): exchange, twiddles, then `nside` side arrays of
// Wc x C complex values (Omega rows of the block's columns: coil map, rho, drho, r).
struct ColSmem {
  size_t xch, tw, side, total;
  int nside;
};
__host__ __device__ inline ColSmem col_smem(int mode, int N, int C, int sm_lane, int Wc) {
  ColSmem L{};
  L.nside = (mode == COL_IFFT_PROD_FFT) ? 4 : (mode == COL_IFFT_ADJ_FFT) ? 2 : 0;
  L.xch = 0;
  L.tw = align16((size_t)C * sm_lane * 8);
  L.side = L.tw + align16((size_t)2 * N * 8);
  L.total = L.side + (size_t)L.nside * Wc * C * 8;
  return L;
}

template <int N1, int N2, int CC = NLV_COL_C> struct ColCfg {
  using S = Split<N1, N2>;
  static constexpr int C = CC;                      // adjacent compact columns per block
  static constexpr int THREADS = C * S::TL;
  static_assert(C % 2 == 0, "column staging copies pairs of complex values");
};

// Stages Omega rows of C columns starting at compact column cc0 of a compact (Wc x Wc per coil) array.  A thread
// keeps one 16-byte pair of columns (blockDim.x is a multiple of C/2) and steps down the rows.
__device__ __forceinline__ void stage_compact_cols(float2* sdst, const float2* plane, int cc0, int C, int Wc) {
  const int cpr = C / 2;                               // 16-byte chunks per row segment
  const int k = threadIdx.x % cpr, cc = cc0 + 2 * k, step = blockDim.x / cpr;
  if (cc >= Wc) return;
  const float2* src = plane + cc;
  for (int cr = threadIdx.x / cpr; cr < Wc; cr += step) cp_async16(sdst + (size_t)cr * C + 2 * k, src + (size_t)cr * Wc);
}
// Same for a natural N x N plane (rows and columns mapped from compact to natural indices).
__device__ __forceinline__ void stage_natural_cols(float2* sdst, const float2* plane, int cc0, int C, int Wc, int N,
                                                   int f) {
  if ((f & 1) == 0) {                                  // compact pairs (2k, 2k+1) stay adjacent in natural order
    const int cpr = C / 2;
    const int k = threadIdx.x % cpr, cc = cc0 + 2 * k, step = blockDim.x / cpr;
    if (cc >= Wc) return;
    const float2* src = plane + to_natural(cc, N, f);
    for (int cr = threadIdx.x / cpr; cr < Wc; cr += step)
      cp_async16(sdst + (size_t)cr * C + 2 * k, src + (size_t)to_natural(cr, N, f) * N);
  } else {
    for (int i = threadIdx.x; i < Wc * C; i += blockDim.x) {
      const int cr = i / C, k = i % C, cc = cc0 + k;
      if (cc < Wc)
        cp_async8(sdst + (size_t)cr * C + k, plane + (size_t)to_natural(cr, N, f) * N + to_natural(cc, N, f));
    }
  }
}

template <int N1, int N2, int MODE, bool STDF, int CC>
__device__ __forceinline__ void col_stage_side(const KArgs& A, int bid, unsigned char* smem_raw) {
  using S = Split<N1, N2>;
  constexpr int N = S::N, C = ColCfg<N1, N2, CC>::C;
  const int f = STDF ? N / 4 : A.f, Wc = STDF ? N / 2 : A.Wc;
  const int strips = (Wc + C - 1) / C;
  const int j = bid / strips;
  const int cc0 = (bid % strips) * C;
  const ColSmem L = col_smem(MODE, N, C, S::SM_LANE_COL, Wc);
  stage_bytes(smem_raw + L.tw, A.twA, N * 8);
  stage_bytes(smem_raw + L.tw + N * 8, A.twB, N * 8);
  if (j < A.nrows) {
    float2* sd = (float2*)(smem_raw + L.side);
    const size_t sstride = (size_t)Wc * C;
    if constexpr (MODE == COL_IFFT_PROD_FFT || MODE == COL_IFFT_ADJ_FFT) {
      stage_compact_cols(sd, A.coil + (size_t)j * Wc * Wc, cc0, C, Wc);
      stage_natural_cols(sd + sstride, A.rho, cc0, C, Wc, N, f);
    }
    if constexpr (MODE == COL_IFFT_PROD_FFT) {
      stage_natural_cols(sd + 2 * sstride, A.drho, cc0, C, Wc, N, f);
      if (A.pupd) stage_natural_cols(sd + 3 * sstride, A.r, cc0, C, Wc, N, f);
    }
  }
}

// prestaged: the twiddles and side inputs were staged by col_stage_side before the dependent-launch wait.
template <int N1, int N2, int MODE, bool STDF = false, class TC = NoTc, int CC = NLV_COL_C>
__device__ __forceinline__ void col_pass_body(const KArgs& A, int bid, unsigned char* smem_raw, TC* tc = nullptr,
                                              bool prestaged = false) {
  using S = Split<N1, N2>;
  constexpr int N = S::N, E = S::E, C = ColCfg<N1, N2, CC>::C;
  const int lane = threadIdx.x % C, idx = threadIdx.x / C;
  const int f = STDF ? N / 4 : A.f, Wc = STDF ? N / 2 : A.Wc;
  const int strips = (Wc + C - 1) / C;
  const int j = bid / strips;
  const int cc0 = (bid % strips) * C;
  const int cc = cc0 + lane;
  const bool active = cc < Wc && j < A.nrows;
  const int x2 = to_natural(cc, N, f);
  const ColSmem L = col_smem(MODE, N, C, S::SM_LANE_COL, Wc);
  float2* sm = (float2*)(smem_raw + L.xch) + lane * S::SM_LANE_COL;
  const float2* twA = (const float2*)(smem_raw + L.tw);
  const float2* twB = twA + N;
  const float2* side = (const float2*)(smem_raw + L.side);
  const float rs = rsqrtf((float)N);
  const size_t tbase = (size_t)j * N * Wc + cc;       // T element (row e1) at tbase + e1*Wc
  const size_t cbase = (size_t)j * Wc * Wc + cc;      // compact coil element (row cr) at cbase + cr*Wc
  float2 v[E];

  // ---- main loads, layout A: thread a < N1 holds column elements a + N1*m
  if (idx < N1) {
#pragma unroll
    for (int m = 0; m < N2; ++m) {
      const int e1 = idx + N1 * m;
      float2 val = make_float2(0.f, 0.f);
      if constexpr (MODE == COL_PROD_FFT || MODE == COL_SIM_FFT) {
        if (active && in_omega(e1, N, f)) {
          const float2 c = (MODE == COL_PROD_FFT) ? A.coil[cbase + (size_t)to_compact(e1, N, f) * Wc]
                                                  : A.cimg[((size_t)j * N + e1) * N + x2];
          val = cmul(A.rho[(size_t)e1 * N + x2], c);
        }
      } else {
        if (active) val = A.src[tbase + (size_t)e1 * Wc];
      }
      v[m] = val;
    }
  }
  // ---- staged side inputs (Omega rows of this block's columns) and twiddles
  if (!prestaged) col_stage_side<N1, N2, MODE, STDF, CC>(A, bid, smem_raw);
  cp_async_wait_all();
  __syncthreads();

  if constexpr (MODE == COL_PROD_FFT || MODE == COL_SIM_FFT) {
    fft_AtoB<N1, N2, -1, false>(v, sm, twA, idx, tc);
    if (active && idx < N2) {
#pragma unroll
      for (int m = 0; m < N1; ++m) {
        const int e1 = idx + N2 * m;
        A.dst[tbase + (size_t)e1 * Wc] = cscale(v[m], rs);
      }
    }
    return;
  } else {
    fft_AtoB<N1, N2, +1, MODE != COL_IFFT_C>(v, sm, twA, idx, tc);
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
      const size_t sstride = (size_t)Wc * C;
      const float beta = (MODE == COL_IFFT_PROD_FFT && A.pupd) ? cg_beta(A) : 0.f;
      if (idx < N2) {
#pragma unroll
        for (int m = 0; m < N1; ++m) {
          const int e1 = idx + N2 * m;
          float2 out = make_float2(0.f, 0.f);
          if (active && in_omega(e1, N, f)) {
            const int cr = to_compact(e1, N, f);
            const float2 u = cscale(v[m], rs);
            const float2 c = side[(size_t)cr * C + lane];
            const float2 rh = side[sstride + (size_t)cr * C + lane];
            if constexpr (MODE == COL_IFFT_PROD_FFT) {
              float2 dr = side[2 * sstride + (size_t)cr * C + lane];
              if (A.pupd) {          // rho part of p = r + beta p (written later by the last row pass)
                const float2 rv = side[3 * sstride + (size_t)cr * C + lane];
                dr = make_float2(fmaf(beta, dr.x, rv.x), fmaf(beta, dr.y, rv.y));
              }
              out = cadd(cmul(dr, c), cmul(rh, u));
            } else {  // COL_IFFT_ADJ_FFT
              A.zsum[cbase + (size_t)cr * Wc] = cmulc(c, u);
              out = cmulc(rh, u);
            }
          }
          v[m] = out;
        }
      }
      // without its closing barrier the DF^H pass (100 -> 92 registers) measured 1.1 us slower at 384^2/10
      fft_AtoB<N2, N1, -1, MODE == COL_IFFT_ADJ_FFT>(v, sm, twB, idx, tc);
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

template <int N1, int N2, int MODE, bool STDF = false, int CC = NLV_COL_C>
__global__ void __launch_bounds__(ColCfg<N1, N2, CC>::THREADS) col_pass(const KArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int early = cg_flags_early(A);
  // before the wait only through L2 (16-byte copies): an odd f stages the natural planes with 8-byte copies,
  // which go through L1, after the wait
  const bool pre = STDF || (A.f & 1) == 0;
  if (pre) col_stage_side<N1, N2, MODE, STDF, CC>(A, blockIdx.x, smem_raw);
  pdl_enter();
  if (cg_stopped_after(A, early)) {
    cp_async_wait_all();
    return;
  }
  col_pass_body<N1, N2, MODE, STDF, NoTc, CC>(A, blockIdx.x, smem_raw, nullptr, pre);
}

// ------------------------------------------------------------------------------- tensor-core passes ----
// The same passes with their radix-16 DFT stages on the tensor cores (tc_dft.cuh): the engine's shared memory
// follows the pass's own layout (offset tc_offset(...) below), its TMEM is allocated after the dependent-launch
// wait and freed at the end.
__host__ __device__ constexpr size_t tc_offset(size_t pass_bytes) { return (pass_bytes + 127) / 128 * 128; }

template <int N1, int N2, int MODE, bool STDF>
__global__ void __launch_bounds__(kRowMaxThreads, 1) row_pass_tc(const KArgs A) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  pdl_enter();
  if (cg_stopped(A)) return;
  using S = Split<N1, N2>;
  const RowSmem L = row_smem(MODE, S::N, blockDim.x / S::TL, S::SM_LANE);
  TcDft tc;
  tc.setup(smem_raw + tc_offset(L.total), A.tcB, &A.sc->flags);
  row_pass_body<N1, N2, MODE, STDF, TcDft>(A, blockIdx.x, gridDim.x, smem_raw, &tc);
  tc.teardown();
}

template <int N1, int N2, int MODE, bool STDF>
__global__ void __launch_bounds__(ColCfg<N1, N2>::THREADS, 1) col_pass_tc(const KArgs A) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  pdl_enter();
  if (cg_stopped(A)) return;
  using S = Split<N1, N2>;
  const ColSmem L = col_smem(MODE, S::N, ColCfg<N1, N2>::C, S::SM_LANE_COL, STDF ? S::N / 2 : A.Wc);
  TcDft tc;
  tc.setup(smem_raw + tc_offset(L.total), A.tcB, &A.sc->flags);
  col_pass_body<N1, N2, MODE, STDF, TcDft>(A, blockIdx.x, smem_raw, &tc);
  tc.teardown();
}

// --------------------------------------------------------------------------------------------- batches ----
// A batched launch runs one pass for several independent frames of the same grid side: frame f owns the blocks
// [first[f], first[f+1]) and its own arguments args[f] (pointers into its own workspace).  Each block finds its
// frame, copies that frame's arguments into shared memory and runs the same pass body as a single-frame launch.
struct BatchArgs {
  const KArgs* args;       // per-frame arguments (device)
  const int* first;        // nframes + 1 block offsets (device)
  int nframes;
  int total;               // work items = first[nframes]; a block takes items blockIdx.x, + gridDim.x, ...
};

// Work item w of a batched launch: its frame's arguments (copied to shared memory), its block index within the
// frame and the frame's block count.  Every thread of the block calls it (barriers).
__device__ __forceinline__ const KArgs& batch_frame(const BatchArgs& B, int w, int& bid, int& nblk) {
  __shared__ KArgs sa;
  __shared__ int sf, sb, sn;
  __syncthreads();         // the previous work item of this block is done with sa
  // the frame is the number of block offsets first[1 .. nframes-1] at or below this item (offsets increase):
  // the first warp tests 32 of them per step, all loads of a step in flight together
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x, nl = warp_lanes();
    const unsigned live = nl >= 32 ? 0xffffffffu : (1u << nl) - 1u;
    int f = 0;
    for (int base = 1; base < B.nframes; base += nl) {
      const int k = base + lane;
      const bool le = lane < nl && k < B.nframes && B.first[k] <= w;
      f += __popc(__ballot_sync(live, le));
    }
    if (lane == 0) {
      sf = f;
      sb = w - B.first[f];
      sn = B.first[f + 1] - B.first[f];
    }
  }
  __syncthreads();
  const int* src = (const int*)(B.args + sf);
  for (int i = threadIdx.x; i < (int)(sizeof(KArgs) / sizeof(int)); i += blockDim.x) ((int*)&sa)[i] = src[i];
  bid = sb;
  nblk = sn;
  __syncthreads();
  return sa;
}

template <int N1, int N2, int MODE, bool STDF = false>
__global__ void __launch_bounds__(kRowMaxThreads, kRowCtasPerSM) row_pass_batch(const BatchArgs B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_enter();
  for (int w = blockIdx.x; w < B.total; w += gridDim.x) {
    int bid, nblk;
    const KArgs& A = batch_frame(B, w, bid, nblk);
    if (cg_stopped(A)) continue;
    row_pass_body<N1, N2, MODE, STDF>(A, bid, nblk, smem_raw);
  }
}

template <int N1, int N2, int MODE, bool STDF = false>
__global__ void __launch_bounds__(ColCfg<N1, N2>::THREADS) col_pass_batch(const BatchArgs B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_enter();
  for (int w = blockIdx.x; w < B.total; w += gridDim.x) {
    int bid, nblk;
    const KArgs& A = batch_frame(B, w, bid, nblk);
    if (cg_stopped(A)) continue;
    col_pass_body<N1, N2, MODE, STDF>(A, bid, smem_raw);
  }
}

// ------------------------------------------------------------------------- batches of several sides ----
// One launch per pass for frames of every grid side in kMultiSides: the block dispatches on its work item's grid
// side to that side's pass body.  Row passes run kRowMaxThreads threads (kRowMaxThreads / TL whole lanes of the
// side, the rest idle), column passes kMultiColThreads (NLV_COL_C columns x the largest lane width).
constexpr int kMultiSides[] = {128, 192, 256, 320, 384};
constexpr int kNumMultiSides = 5;
constexpr int kMultiColThreads = NLV_COL_C * 24;
__host__ __device__ constexpr bool multi_side(int n) {
  return n == 128 || n == 192 || n == 256 || n == 320 || n == 384;
}

// Each side's body is a separate (not inlined) function, so that registers are allocated per side rather than
// across all sides' branches at once.
template <int N1, int N2, int MODE, bool STDF>
__device__ __noinline__ void row_body_call(const KArgs& A, int bid, int nblk, unsigned char* smem) {
  row_pass_body<N1, N2, MODE, STDF>(A, bid, nblk, smem);
}
template <int N1, int N2, int MODE, bool STDF>
__device__ __noinline__ void col_body_call(const KArgs& A, int bid, unsigned char* smem) {
  col_pass_body<N1, N2, MODE, STDF>(A, bid, smem);
}
template <int MODE, bool STDF>
__device__ __forceinline__ void row_body_of_side(const KArgs& A, int bid, int nblk, unsigned char* smem) {
  switch (A.N) {
    case 128: row_body_call<8, 16, MODE, STDF>(A, bid, nblk, smem); break;
    case 192: row_body_call<12, 16, MODE, STDF>(A, bid, nblk, smem); break;
    case 256: row_body_call<16, 16, MODE, STDF>(A, bid, nblk, smem); break;
    case 320: row_body_call<16, 20, MODE, STDF>(A, bid, nblk, smem); break;
    default: row_body_call<16, 24, MODE, STDF>(A, bid, nblk, smem); break;
  }
}
template <int MODE, bool STDF>
__device__ __forceinline__ void col_body_of_side(const KArgs& A, int bid, unsigned char* smem) {
  switch (A.N) {
    case 128: col_body_call<8, 16, MODE, STDF>(A, bid, smem); break;
    case 192: col_body_call<12, 16, MODE, STDF>(A, bid, smem); break;
    case 256: col_body_call<16, 16, MODE, STDF>(A, bid, smem); break;
    case 320: col_body_call<16, 20, MODE, STDF>(A, bid, smem); break;
    default: col_body_call<16, 24, MODE, STDF>(A, bid, smem); break;
  }
}

template <int MODE, bool STDF>
__global__ void __launch_bounds__(kRowMaxThreads, kRowCtasPerSM) row_pass_multi(const BatchArgs B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_enter();
  for (int w = blockIdx.x; w < B.total; w += gridDim.x) {
    int bid, nblk;
    const KArgs& A = batch_frame(B, w, bid, nblk);
    if (cg_stopped(A)) continue;
    row_body_of_side<MODE, STDF>(A, bid, nblk, smem_raw);
  }
}

template <int MODE, bool STDF>
__global__ void __launch_bounds__(kMultiColThreads) col_pass_multi(const BatchArgs B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_enter();
  for (int w = blockIdx.x; w < B.total; w += gridDim.x) {
    int bid, nblk;
    const KArgs& A = batch_frame(B, w, bid, nblk);
    if (cg_stopped(A)) continue;
    col_body_of_side<MODE, STDF>(A, bid, smem_raw);
  }
}

// The multi-side kernels of every pass (defined in batch_multi.cu) and their dynamic shared memory (the largest
// over the sides).
struct MultiKernels {
  const void* row[NUM_ROW_MODES];
  const void* row_std[NUM_ROW_MODES];
  const void* col[NUM_COL_MODES];
  const void* col_std[NUM_COL_MODES];
  size_t row_smem[NUM_ROW_MODES];
  size_t col_smem[NUM_COL_MODES];
};
const MultiKernels* multi_kernels();

// ------------------------------------------------------------------------------- per-size kernel table ----
struct SizeKernels {
  int N1, N2;
  int tl;                   // threads per lane
  int col_lanes, col_threads;
  int sm_lane;              // shared float2 per lane for one exchange (row passes)
  int sm_lane_col;          // the same for column passes (bank-conflict padding)
  const void* row[NUM_ROW_MODES];
  const void* col[NUM_COL_MODES];
  const void* row_batch[NUM_ROW_MODES];
  const void* col_batch[NUM_COL_MODES];
  // Passes of the CG iteration specialised for the standard field of view f = N/4 (a compile-time constant, so
  // the Omega tests of the register-held elements fold away); nullptr where the generic kernel is used.
  const void* row_std[NUM_ROW_MODES];
  const void* col_std[NUM_COL_MODES];
  const void* row_std_batch[NUM_ROW_MODES];
  const void* col_std_batch[NUM_COL_MODES];
  // Passes with their radix-16 DFT stages on the tensor cores (sides whose split has a factor 16); nullptr where
  // not compiled.  row_tc_std / col_tc_std: the standard-field-of-view forms, as row_std / col_std.
  const void* row_tc[NUM_ROW_MODES];
  const void* col_tc[NUM_COL_MODES];
  const void* row_tc_std[NUM_ROW_MODES];
  const void* col_tc_std[NUM_COL_MODES];
  size_t row_smem(int mode, int lanes) const { return nlv::row_smem(mode, N1 * N2, lanes, sm_lane).total; }
  size_t col_smem(int mode, int Wc) const { return nlv::col_smem(mode, N1 * N2, col_lanes, sm_lane_col, Wc).total; }
  size_t row_smem_tc(int mode, int lanes) const { return tc_offset(row_smem(mode, lanes)) + tc_smem_bytes(lanes * tl); }
  size_t col_smem_tc(int mode, int Wc) const { return tc_offset(col_smem(mode, Wc)) + tc_smem_bytes(col_threads); }
};

// Launch geometry of a row pass: `blocks` blocks of `lanes` lanes, each taking rows_per_cta rows (and rho_per_cta
// pixels of the rho plane when the pass has one), so that the rows are split evenly over ctas_per_sm blocks per SM.
struct RowGrid {
  int blocks, lanes, rows_per_cta, rho_per_cta;
};
inline RowGrid row_grid(const SizeKernels* k, int nrows, long rho_pixels, int sms, int ctas_per_sm) {
  RowGrid g{};
  const int max_lanes = kRowMaxThreads / k->tl;
  int want = sms * ctas_per_sm;
  if (want > nrows) want = nrows;
  const int per = (nrows + want - 1) / want;
  const int rounds = (per + max_lanes - 1) / max_lanes;
  g.lanes = (per + rounds - 1) / rounds;
  g.rows_per_cta = per;
  g.blocks = (nrows + per - 1) / per;
  g.rho_per_cta = (int)((rho_pixels + g.blocks - 1) / g.blocks);
  return g;
}

// Tuning variants of a side (nlinv_autotune): the default table with other column-strip widths, and the single-frame
// passes of an alternative four-step split.  They hold no batch or tensor-core kernels.
template <int N1, int N2, int CC> SizeKernels make_size_kernels_strip(const SizeKernels& base) {
  SizeKernels s = base;
  s.col_lanes = ColCfg<N1, N2, CC>::C;
  s.col_threads = ColCfg<N1, N2, CC>::THREADS;
  s.col[COL_IFFT_C] = (const void*)col_pass<N1, N2, COL_IFFT_C, false, CC>;
  s.col[COL_PROD_FFT] = (const void*)col_pass<N1, N2, COL_PROD_FFT, false, CC>;
  s.col[COL_SIM_FFT] = (const void*)col_pass<N1, N2, COL_SIM_FFT, false, CC>;
  s.col[COL_IFFT_PROD_FFT] = (const void*)col_pass<N1, N2, COL_IFFT_PROD_FFT, false, CC>;
  s.col[COL_IFFT_ADJ_FFT] = (const void*)col_pass<N1, N2, COL_IFFT_ADJ_FFT, false, CC>;
  for (int m = 0; m < NUM_COL_MODES; ++m) s.col_std[m] = nullptr;
  s.col_std[COL_IFFT_PROD_FFT] = (const void*)col_pass<N1, N2, COL_IFFT_PROD_FFT, true, CC>;
  for (int m = 0; m < NUM_ROW_MODES; ++m) s.row_batch[m] = s.row_std_batch[m] = s.row_tc[m] = s.row_tc_std[m] = nullptr;
  for (int m = 0; m < NUM_COL_MODES; ++m) s.col_batch[m] = s.col_std_batch[m] = s.col_tc[m] = s.col_tc_std[m] = nullptr;
  return s;
}

template <int N1, int N2> SizeKernels make_size_kernels_single() {
  SizeKernels s{};
  s.N1 = N1;
  s.N2 = N2;
  s.tl = Split<N1, N2>::TL;
  s.col_lanes = ColCfg<N1, N2>::C;
  s.col_threads = ColCfg<N1, N2>::THREADS;
  s.sm_lane = Split<N1, N2>::SM_LANE;
  s.sm_lane_col = Split<N1, N2>::SM_LANE_COL;
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
  s.row_std[ROW_W_IFFT] = (const void*)row_pass<N1, N2, ROW_W_IFFT, true>;
  s.row_std[ROW_PSF] = (const void*)row_pass<N1, N2, ROW_PSF, true>;
  s.row_std[ROW_FFT_W_NORMAL] = (const void*)row_pass<N1, N2, ROW_FFT_W_NORMAL, true>;
  s.col_std[COL_IFFT_PROD_FFT] = (const void*)col_pass<N1, N2, COL_IFFT_PROD_FFT, true>;
  return s;
}

template <int N1, int N2> SizeKernels make_size_kernels() {
  SizeKernels s{};
  s.N1 = N1;
  s.N2 = N2;
  s.tl = Split<N1, N2>::TL;
  s.col_lanes = ColCfg<N1, N2>::C;
  s.col_threads = ColCfg<N1, N2>::THREADS;
  s.sm_lane = Split<N1, N2>::SM_LANE;
  s.sm_lane_col = Split<N1, N2>::SM_LANE_COL;
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
  s.row_batch[ROW_W_IFFT] = (const void*)row_pass_batch<N1, N2, ROW_W_IFFT>;
  s.row_batch[ROW_PSF] = (const void*)row_pass_batch<N1, N2, ROW_PSF>;
  s.row_batch[ROW_FFT_P_OUT] = (const void*)row_pass_batch<N1, N2, ROW_FFT_P_OUT>;
  s.row_batch[ROW_FFT_RESID] = (const void*)row_pass_batch<N1, N2, ROW_FFT_RESID>;
  s.row_batch[ROW_P_IFFT] = (const void*)row_pass_batch<N1, N2, ROW_P_IFFT>;
  s.row_batch[ROW_FFT_W_ADJ] = (const void*)row_pass_batch<N1, N2, ROW_FFT_W_ADJ>;
  s.row_batch[ROW_FFT_W_NORMAL] = (const void*)row_pass_batch<N1, N2, ROW_FFT_W_NORMAL>;
  s.row_batch[ROW_FFT_W_RHS] = (const void*)row_pass_batch<N1, N2, ROW_FFT_W_RHS>;
  s.col_batch[COL_IFFT_C] = (const void*)col_pass_batch<N1, N2, COL_IFFT_C>;
  s.col_batch[COL_PROD_FFT] = (const void*)col_pass_batch<N1, N2, COL_PROD_FFT>;
  s.col_batch[COL_SIM_FFT] = (const void*)col_pass_batch<N1, N2, COL_SIM_FFT>;
  s.col_batch[COL_IFFT_PROD_FFT] = (const void*)col_pass_batch<N1, N2, COL_IFFT_PROD_FFT>;
  s.col_batch[COL_IFFT_ADJ_FFT] = (const void*)col_pass_batch<N1, N2, COL_IFFT_ADJ_FFT>;
  // measured: the p-update, PSF and normal-operator row passes and the DF column pass gain from the constant
  // field of view (the batched p-update pass also stops spilling); the DF^H column pass does not
  s.row_std[ROW_W_IFFT] = (const void*)row_pass<N1, N2, ROW_W_IFFT, true>;
  s.row_std[ROW_PSF] = (const void*)row_pass<N1, N2, ROW_PSF, true>;
  s.row_std[ROW_FFT_W_NORMAL] = (const void*)row_pass<N1, N2, ROW_FFT_W_NORMAL, true>;
  s.col_std[COL_IFFT_PROD_FFT] = (const void*)col_pass<N1, N2, COL_IFFT_PROD_FFT, true>;
  s.row_std_batch[ROW_W_IFFT] = (const void*)row_pass_batch<N1, N2, ROW_W_IFFT, true>;
  s.row_std_batch[ROW_PSF] = (const void*)row_pass_batch<N1, N2, ROW_PSF, true>;
  s.row_std_batch[ROW_FFT_W_NORMAL] = (const void*)row_pass_batch<N1, N2, ROW_FFT_W_NORMAL, true>;
  s.col_std_batch[COL_IFFT_PROD_FFT] = (const void*)col_pass_batch<N1, N2, COL_IFFT_PROD_FFT, true>;
  return s;
}

// The kernel table of a side whose split has a factor 16, with the tensor-core passes added.
template <int N1, int N2> SizeKernels make_size_kernels_tc() {
  static_assert(N1 == 16 || N2 == 16, "the tensor-core stage is a radix-16 DFT");
  SizeKernels s = make_size_kernels<N1, N2>();
  s.row_tc[ROW_W_IFFT] = (const void*)row_pass_tc<N1, N2, ROW_W_IFFT, false>;
  s.row_tc[ROW_PSF] = (const void*)row_pass_tc<N1, N2, ROW_PSF, false>;
  s.row_tc[ROW_FFT_P_OUT] = (const void*)row_pass_tc<N1, N2, ROW_FFT_P_OUT, false>;
  s.row_tc[ROW_FFT_RESID] = (const void*)row_pass_tc<N1, N2, ROW_FFT_RESID, false>;
  s.row_tc[ROW_P_IFFT] = (const void*)row_pass_tc<N1, N2, ROW_P_IFFT, false>;
  s.row_tc[ROW_FFT_W_ADJ] = (const void*)row_pass_tc<N1, N2, ROW_FFT_W_ADJ, false>;
  s.row_tc[ROW_FFT_W_NORMAL] = (const void*)row_pass_tc<N1, N2, ROW_FFT_W_NORMAL, false>;
  s.row_tc[ROW_FFT_W_RHS] = (const void*)row_pass_tc<N1, N2, ROW_FFT_W_RHS, false>;
  s.col_tc[COL_IFFT_C] = (const void*)col_pass_tc<N1, N2, COL_IFFT_C, false>;
  s.col_tc[COL_PROD_FFT] = (const void*)col_pass_tc<N1, N2, COL_PROD_FFT, false>;
  s.col_tc[COL_SIM_FFT] = (const void*)col_pass_tc<N1, N2, COL_SIM_FFT, false>;
  s.col_tc[COL_IFFT_PROD_FFT] = (const void*)col_pass_tc<N1, N2, COL_IFFT_PROD_FFT, false>;
  s.col_tc[COL_IFFT_ADJ_FFT] = (const void*)col_pass_tc<N1, N2, COL_IFFT_ADJ_FFT, false>;
  s.row_tc_std[ROW_PSF] = (const void*)row_pass_tc<N1, N2, ROW_PSF, true>;
  s.row_tc_std[ROW_FFT_W_NORMAL] = (const void*)row_pass_tc<N1, N2, ROW_FFT_W_NORMAL, true>;
  s.col_tc_std[COL_IFFT_PROD_FFT] = (const void*)col_pass_tc<N1, N2, COL_IFFT_PROD_FFT, true>;
  return s;
}

}  // namespace nlv
