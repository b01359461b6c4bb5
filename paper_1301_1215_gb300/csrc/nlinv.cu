// C interface, context and solver driver of the GB300 NLINV library (declared in include/nlinv.h).
//
// The driver queues the pass kernels of kernels.cuh on the context's stream:
//   coil maps      c_j = W^-1 chat_j on Omega                  row ROW_W_IFFT, col COL_IFFT_C
//   F x            P FFT(M rho c_j)                            col COL_PROD_FFT, row ROW_FFT_P_OUT / ROW_FFT_RESID
//   DF dx          P FFT(M (drho c_j + rho W^-1 dchat_j))       row ROW_W_IFFT, col COL_IFFT_PROD_FFT, row ROW_FFT_P_OUT
//   DF^H r         (sum_j conj(c_j) z_j, w FFT(conj(rho) z_j)) row ROW_P_IFFT, col COL_IFFT_ADJ_FFT, row ROW_FFT_W_ADJ
//   (DF^H DF + alpha) p   the PSF form of Sec. 3.1: row ROW_W_IFFT, col COL_IFFT_PROD_FFT, row ROW_PSF,
//                         col COL_IFFT_ADJ_FFT, row ROW_FFT_W_NORMAL (+ Re<p, q>)
//   CG updates     dx += alpha p, r -= alpha q (+ |r|^2); p = r + beta p
// Each operator application performs the two 2D transforms per operator of Table 1, batched over all coils.
// Beyond the paper's method: the gradient through the reconstruction (nlinv_reconstruct_checkpoints and
// nlinv_reconstruct_vjp: the same operators at other linearisation points, plus a CG solve per Newton step),
// batches of independent frames (nlinv_batch_*: the same passes, one launch per grid side), and the launch-shape
// autotuner (nlinv_autotune: whole graph-replayed frames per candidate).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "nlinv.h"
#include "sizes.cuh"

using nlv::KArgs;
using nlv::Scalars;
using nlv::SizeKernels;

namespace {

thread_local std::string g_create_error;

// ------------------------------------------------------------------------------------------ vector kernels ----
// float4 groups of CG-step operands in flight per thread.  Two keep the kernel at 64 registers, four blocks of 256
// threads per SM; four groups need 96 registers (two blocks per SM, measured 13.2 against 11.5 us per step at
// 384 x 384 with 10 coils) or spill at 64.
constexpr int kCgGroups = 2;
// dx += alpha p; r -= alpha q; partial of |r|^2 -> rr_part[bid], over this block's share of the A.n2 float4.
// A thread sums the squares of at most two float4 (8 products) in FP32 before adding them to its FP64 partial.
__device__ __forceinline__ void cg_step_update(float4& d, float4& r, const float4& p, const float4& q, float a,
                                               float& acc) {
  d.x = fmaf(a, p.x, d.x); d.y = fmaf(a, p.y, d.y); d.z = fmaf(a, p.z, d.z); d.w = fmaf(a, p.w, d.w);
  r.x = fmaf(-a, q.x, r.x); r.y = fmaf(-a, q.y, r.y); r.z = fmaf(-a, q.z, r.z); r.w = fmaf(-a, q.w, r.w);
  acc += r.x * r.x + r.y * r.y + r.z * r.z + r.w * r.w;
}

// The CG step's scalars, the same in every block: t = Re<p, A p> from the n_pq partials, alpha = |r|^2 / t, and the
// rounding-floor test (see cg_step_body).  Block 0 publishes them; s_alpha and s_skip (stopped by an earlier
// iteration) are valid for every thread of the block on return.
__device__ __forceinline__ void cg_step_decide(const KArgs& A, int bid, float& s_alpha, int& s_skip, double* red) {
  double t = 0.0;
  for (int k = threadIdx.x; k < A.n_pq; k += blockDim.x) t += A.pq_part[k];
  t = nlv::block_sum(t, red);
  if (threadIdx.x == 0) {
    const double rr = A.sc->rr;
    const int flags = *(volatile int*)&A.sc->flags;
    const bool was_stopped = (flags & nlv::kFlagCgStopped) != 0;
    double a = 0.0;
    bool stop = false;
    if (!was_stopped) {
      if (!isfinite(t) || !isfinite(rr)) {
        if (bid == 0) A.sc->flags |= nlv::kFlagBreakdown;
        stop = true;
      } else if (rr > nlv::kCgFloor2 * A.sc->rr0 && t > 0.0) {
        a = rr / t;
      } else {
        stop = true;
      }
    }
    if (bid == 0) {
      A.sc->pq = t;
      A.sc->alpha = a;
      A.sc->rr_prev = rr;
      if (stop) {
        A.sc->flags |= nlv::kFlagCgStopped;
        A.sc->cg_stop[A.slot] = A.iter;
      }
    }
    s_alpha = (float)a;
    s_skip = was_stopped ? 1 : 0;     // stopped by an earlier iteration: nothing to update
  }
  __syncthreads();
}

template <int G = 2>
__device__ __forceinline__ void cg_step_body(const KArgs& A, int bid, int nblk) {
  const float4* __restrict__ p4 = (const float4*)A.p;
  const float4* __restrict__ q4 = (const float4*)A.q;
  float4* __restrict__ r4 = (float4*)A.r;
  float4* __restrict__ dx4 = (float4*)A.dx;
  // Two groups of operands per thread in flight: the first two are loaded while the block forms
  // alpha = |r|^2 / Re<p, A p> from the partials of the normal-operator pass (every block sums them in the same
  // fixed order).  The solve stops at the rounding floor: |r|^2 <= kCgFloor2 |b|^2 (|r| at the FP32 unit roundoff
  // relative to |b|, including b = 0), Re<p, A p> <= 0 (impossible in exact arithmetic for the positive definite
  // system of Eq. 3) or a non-finite value.  This step and every later step of the same solve are then empty
  // (alpha = 0), through a flag latched in the scalars until the next right-hand side, and block 0 records the
  // iteration.  Non-finite values also set the breakdown flag.  Every block takes the same decision from the same
  // partials, so a block that already sees the flag set by block 0 in this launch decides as block 0 did.
  const long stride = (long)nblk * blockDim.x;
  long i = bid * (long)blockDim.x + threadIdx.x;
  float4 pg[G], qg[G], rg[G], dg[G];
#pragma unroll
  for (int g = 0; g < G; ++g)
    if (i + g * stride < A.n2) {
      const long k = i + g * stride;
      pg[g] = p4[k]; qg[g] = q4[k]; rg[g] = r4[k]; dg[g] = dx4[k];
    }
  __shared__ float s_alpha;
  __shared__ int s_skip;
  __shared__ double red[32];
  cg_step_decide(A, bid, s_alpha, s_skip, red);
  if (s_skip) return;                 // the same for the whole block (thread 0 decided for it)
  const float a = s_alpha;
  double accd = 0.0;
  // G groups in flight per thread; each group's operands for the next round are loaded right after it is stored,
  // while the other groups of this round are processed
  while (i < A.n2) {
    float acc = 0.f;
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const long k = i + g * stride;
      if (k < A.n2) {
        cg_step_update(dg[g], rg[g], pg[g], qg[g], a, acc);
        dx4[k] = dg[g];
        r4[k] = rg[g];
        const long kn = k + G * stride;
        if (kn < A.n2) { pg[g] = p4[kn]; qg[g] = q4[kn]; rg[g] = r4[kn]; dg[g] = dx4[kn]; }
      }
    }
    accd += (double)acc;
    i += G * stride;
  }
  const double s = nlv::block_sum(accd, red);
  if (threadIdx.x == 0) A.rr_part[bid] = s;
}

// ------------------------------------------------------------------ CG step with bulk asynchronous copies ----
// The single-frame CG step as a persistent kernel, one block per SM: the vector is cut into chunks of kBulkChunk
// float4 per array, and a block's chunks (b, b + nblk, ...) stream p, q, r and dx through a ring of kBulkStages
// shared-memory stages filled by cp.async.bulk (one thread issues four bulk copies per chunk, completion counted in
// bytes on the stage's mbarrier), so that up to kBulkStages chunks -- 3 x 64 KB -- are in flight per SM without
// holding them in registers.  Each thread then updates its share of the chunk from shared memory and stores dx and
// r directly.  Every wait is bounded (about a second of clock cycles): on a timeout the kernel sets
// kFlagCopyTimeout, waits once more (bounded) for its copies in flight and returns; the host reports ECUDA.
constexpr int kBulkThreads = 512;
constexpr int kBulkChunk = 1024;        // float4 per array per chunk (16 KB)
constexpr int kBulkStages = 3;
constexpr size_t kBulkSmem = (size_t)kBulkStages * 4 * kBulkChunk * sizeof(float4) + kBulkStages * 8;
constexpr int kFlagCopyTimeout = 8;     // Scalars::flags bit: a bulk-copy completion wait timed out

__device__ __forceinline__ uint32_t shared_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Waits (bounded by about a second of clock cycles) for the phase of parity `parity` of the mbarrier at bar.
__device__ __forceinline__ bool bulk_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    if (ok) return true;
    if (clock64() - t0 > 2000000000LL) return false;
    __nanosleep(20);
  }
}

// Bytes per array of chunk c.
__device__ __forceinline__ uint32_t bulk_bytes(const KArgs& A, long c) {
  const long off = c * kBulkChunk;
  return (uint32_t)(((A.n2 - off) < kBulkChunk ? (A.n2 - off) : kBulkChunk) * sizeof(float4));
}
// Thread 0: the stage's barrier expects the four arrays of chunk c (one arrival with their byte count).
__device__ __forceinline__ void bulk_expect(const KArgs& A, uint32_t bar, long c) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}"
               ::"r"(bar), "r"(4u * bulk_bytes(A, c)) : "memory");
}
// Thread 0: array a (0 p, 1 q, 2 r, 3 dx) of chunk c into stage s, completion counted on the stage's barrier.
__device__ __forceinline__ void bulk_copy(const KArgs& A, float4* ring, uint32_t bar, long c, int s, int a) {
  const float4* src = (const float4*)(a == 0 ? A.p : a == 1 ? A.q : a == 2 ? A.r : A.dx);
  const uint32_t dst = shared_addr(ring + ((size_t)s * 4 + a) * kBulkChunk);
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src + c * kBulkChunk), "r"(bulk_bytes(A, c)), "r"(bar) : "memory");
}
// Thread 0: chunk c of the four arrays into stage s.
__device__ __forceinline__ void bulk_issue(const KArgs& A, float4* ring, uint32_t bar, long c, int s) {
  bulk_expect(A, bar, c);
#pragma unroll
  for (int a = 0; a < 4; ++a) bulk_copy(A, ring, bar, c, s, a);
}

// With src_early, the first stages' copies of r, dx and of p beyond its rho plane are issued before the
// dependent-launch wait: the kernel before (the normal-operator pass) writes q and the rho plane of p, and r, dx and
// the coil planes of p were written two or more launches back (see cg_flags_early in kernels.cuh); q and the rest
// of p follow the wait.  Without it (back-to-back launches of this kernel alone) every copy follows the wait.
__global__ void __launch_bounds__(kBulkThreads, 1) cg_step_bulk(const KArgs A) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float4* ring = (float4*)smem_raw;
  const uint32_t bar0 = shared_addr(smem_raw + (size_t)kBulkStages * 4 * kBulkChunk * sizeof(float4));
  const int bid = blockIdx.x, nblk = gridDim.x;
  const long nchunks = (A.n2 + kBulkChunk - 1) / kBulkChunk;
  const long mine = bid < nchunks ? (nchunks - bid + nblk - 1) / nblk : 0;   // chunks bid, bid + nblk, ...
  const long rho4 = A.src_early ? (long)A.N * A.N / 2 : A.n2;   // float4 of the rho plane (src_early = 0: all)
  if (threadIdx.x == 0) {
    for (int st = 0; st < kBulkStages; ++st)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8u * st) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const long first = mine < kBulkStages ? mine : kBulkStages;
  if (threadIdx.x == 0) {
    for (long k = 0; k < first; ++k) {
      const long ch = bid + k * nblk;
      const uint32_t bar = bar0 + 8u * (uint32_t)k;
      bulk_expect(A, bar, ch);
      if (A.src_early) {
        bulk_copy(A, ring, bar, ch, (int)k, 2);
        bulk_copy(A, ring, bar, ch, (int)k, 3);
      }
      if (ch * kBulkChunk >= rho4) bulk_copy(A, ring, bar, ch, (int)k, 0);
    }
  }
  nlv::pdl_enter();
  if (threadIdx.x == 0) {
    for (long k = 0; k < first; ++k) {
      const long ch = bid + k * nblk;
      const uint32_t bar = bar0 + 8u * (uint32_t)k;
      bulk_copy(A, ring, bar, ch, (int)k, 1);
      if (ch * kBulkChunk < rho4) bulk_copy(A, ring, bar, ch, (int)k, 0);
      if (!A.src_early) {
        bulk_copy(A, ring, bar, ch, (int)k, 2);
        bulk_copy(A, ring, bar, ch, (int)k, 3);
      }
    }
  }
  __shared__ float s_alpha;
  __shared__ int s_skip;
  __shared__ double red[32];
  cg_step_decide(A, bid, s_alpha, s_skip, red);
  bool timed_out = false;
  if (s_skip) {                       // stopped earlier: let the copies already issued land, then leave
    for (long k = 0; k < first; ++k) bulk_wait(bar0 + 8u * (uint32_t)k, 0);
    return;
  }
  const float a = s_alpha;
  float4* __restrict__ r4 = (float4*)A.r;
  float4* __restrict__ dx4 = (float4*)A.dx;
  double accd = 0.0;
  for (long k = 0; k < mine; ++k) {
    const int st = (int)(k % kBulkStages);
    const uint32_t bar = bar0 + 8u * st;
    if (!bulk_wait(bar, (uint32_t)((k / kBulkStages) & 1))) timed_out = true;
    const long off = (bid + k * nblk) * kBulkChunk;
    const long cnt = (A.n2 - off) < kBulkChunk ? (A.n2 - off) : kBulkChunk;
    const float4* sp = ring + ((size_t)st * 4 + 0) * kBulkChunk;
    const float4* sq = sp + kBulkChunk;
    const float4* sr = sq + kBulkChunk;
    const float4* sd = sr + kBulkChunk;
    float acc = 0.f;
    for (long e = threadIdx.x; e < cnt; e += kBulkThreads) {
      float4 d = sd[e], r = sr[e];
      cg_step_update(d, r, sp[e], sq[e], a, acc);
      dx4[off + e] = d;
      r4[off + e] = r;
    }
    accd += (double)acc;
    __syncthreads();                  // every thread is done with stage st
    if (threadIdx.x == 0 && k + kBulkStages < mine) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      bulk_issue(A, ring, bar, bid + (k + kBulkStages) * nblk, st);
    }
  }
  if (timed_out) {
    if (threadIdx.x == 0) atomicOr(&A.sc->flags, kFlagCopyTimeout);
    for (long k = (mine > kBulkStages ? mine - kBulkStages : 0); k < mine; ++k)
      bulk_wait(bar0 + 8u * (uint32_t)(k % kBulkStages), (uint32_t)((k / kBulkStages) & 1));
  }
  const double sblk = nlv::block_sum(accd, red);
  if (threadIdx.x == 0) A.rr_part[bid] = sblk;
}

// x += dx (x = A.dst)
__device__ __forceinline__ void add_body(const KArgs& A, int bid, int nblk) {
  const float4* __restrict__ d4 = (const float4*)A.dx;
  float4* __restrict__ x4 = (float4*)A.dst;
  for (long i = bid * (long)blockDim.x + threadIdx.x; i < A.n2; i += (long)nblk * blockDim.x) {
    float4 d = d4[i], x = x4[i];
    x.x += d.x; x.y += d.y; x.z += d.z; x.w += d.w;
    x4[i] = x;
  }
}

// Display image rho * sqrt(sum_j |c_j|^2) on Omega, centred: out[i][k] for the signed coordinates (i - f, k - f).
__global__ void image_kernel(const KArgs A) {
  nlv::pdl_enter();
  const int N = A.N, f = A.f, Wc = A.Wc, J = A.J;
  const long total = (long)Wc * Wc;
  for (long o = blockIdx.x * (long)blockDim.x + threadIdx.x; o < total; o += (long)gridDim.x * blockDim.x) {
    const int i = (int)(o / Wc), k = (int)(o % Wc);
    const int cr = (i + f) % Wc, cc = (k + f) % Wc;           // compact indices of the signed coordinates
    float s = 0.f;
    for (int j = 0; j < J; ++j) {
      const float2 c = A.coil[((size_t)j * Wc + cr) * Wc + cc];
      s = fmaf(c.x, c.x, fmaf(c.y, c.y, s));
    }
    const float2 r = A.rho[(size_t)nlv::to_natural(cr, N, f) * N + nlv::to_natural(cc, N, f)];
    A.dst[o] = nlv::cscale(r, sqrtf(s));
  }
}

// 256 threads, at most 64 registers: four blocks fit on an SM (the default vector grid)
template <int G>
__global__ void __launch_bounds__(256, 4) cg_step_kernel(const KArgs A) {
  nlv::pdl_enter();
  cg_step_body<G>(A, blockIdx.x, gridDim.x);
}
__global__ void add_kernel(const KArgs A) {
  nlv::pdl_enter();
  add_body(A, blockIdx.x, gridDim.x);
}
// out = alpha X + coef Y (X = A.src, Y = A.q, out = A.dst) over A.n2 float4
__global__ void axpby_kernel(const KArgs A) {
  nlv::pdl_enter();
  const float4* __restrict__ x4 = (const float4*)A.src;
  const float4* __restrict__ y4 = (const float4*)A.q;
  float4* __restrict__ o4 = (float4*)A.dst;
  const float a = A.alpha, b = A.coef;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < A.n2; i += (long)gridDim.x * blockDim.x) {
    const float4 x = x4[i], y = y4[i];
    o4[i] = make_float4(fmaf(a, x.x, b * y.x), fmaf(a, x.y, b * y.y), fmaf(a, x.z, b * y.z), fmaf(a, x.w, b * y.w));
  }
}

// CG from dx = 0 for the right-hand side b = A.src: r = p = b, dx = 0, |b|^2 -> RED_RR_INIT
__global__ void cg_init_kernel(const KArgs A) {
  nlv::pdl_enter();
  const float4* __restrict__ b4 = (const float4*)A.src;
  float4* __restrict__ r4 = (float4*)A.r;
  float4* __restrict__ p4 = (float4*)A.pout;
  float4* __restrict__ d4 = (float4*)A.dx;
  double acc = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < A.n2; i += (long)gridDim.x * blockDim.x) {
    const float4 b = b4[i];
    r4[i] = b;
    p4[i] = b;
    d4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    acc += (double)(b.x * b.x + b.y * b.y + b.z * b.z + b.w * b.w);
  }
  nlv::grid_reduce(acc, A, blockIdx.x, gridDim.x);
}

// the single-frame CG step
const void* cg_step_fn() { return (const void*)cg_step_kernel<kCgGroups>; }

__global__ void __launch_bounds__(256, 4) cg_step_batch(const nlv::BatchArgs B) {
  nlv::pdl_enter();
  for (int w = blockIdx.x; w < B.total; w += gridDim.x) {
    int bid, nblk;
    const KArgs& A = nlv::batch_frame(B, w, bid, nblk);
    cg_step_body<kCgGroups>(A, bid, nblk);
  }
}
__global__ void add_batch(const nlv::BatchArgs B) {
  nlv::pdl_enter();
  for (int w = blockIdx.x; w < B.total; w += gridDim.x) {
    int bid, nblk;
    const KArgs& A = nlv::batch_frame(B, w, bid, nblk);
    add_body(A, bid, nblk);
  }
}

constexpr int kVecThreads = 256;
constexpr int kTuneVecMax = 8;       // largest vector-kernel blocks per SM that nlinv_autotune tries
constexpr int kTuneMaxCandidates = 16;   // most candidates it times (2 splits + 3 strips + 3 row + 6 vector shapes)
constexpr double kTuneMargin = 0.03; // a candidate replaces the compiled default only when this much faster
#ifndef NLV_VEC_BLOCKS_PER_SM
#define NLV_VEC_BLOCKS_PER_SM 4   // blocks per SM of the vector passes
#endif
constexpr int kProfileKernels = 6;   // kernels of one CG iteration, in the order nlinv_profile_cg reports them

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

// ----------------------------------------------------------------------------------------------- context ----
struct nlinv_ctx {
  nlinv_params prm{};
  int N = 0, J = 0, f = 0, Wc = 0;
  long plane = 0;             // N*N
  long vec = 0;               // (1+J)*N*N complex values of an unknown-space vector
  const SizeKernels* k = nullptr;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  int vec_blocks = 0;         // grid of the vector kernels
  int sms = 0;                // streaming multiprocessors of the device
  int row_ctas_per_sm = nlv::kRowCtasPerSM;   // blocks per SM of the row passes
  // workspace (one allocation)
  void* base = nullptr;
  float2 *x = nullptr, *xref = nullptr, *y = nullptr, *r0 = nullptr;
  float2 *r = nullptr, *p = nullptr, *q = nullptr, *dx = nullptr;
  float2 *T = nullptr, *coil = nullptr, *zsum = nullptr;
  float2 *twA = nullptr, *twB = nullptr;
  float* wtab = nullptr;      // Sobolev weight, N x N
  uint8_t* mask = nullptr;
  double* partials = nullptr;
  double* pq_part = nullptr;  // per-block partials of Re<p, A p> of the normal-operator pass
  double* rr_part = nullptr;  // per-block partials of |r|^2 of the CG step
  Scalars* sc = nullptr;
  // graph of one reconstruction
  cudaGraphExec_t graph = nullptr;
  long graph_launches = 0;
  long launches = 0;
  bool have_state = false;    // a reconstruction has filled the workspace
  int batch_lanes = 0;        // > 0: frame of a batch; row passes use this many lanes and one round per block
  struct Rec {
    const void* fn;
    int grid, block;
    size_t smem;
    KArgs args;
  };
  std::vector<Rec>* rec = nullptr;   // non-null: launches are recorded instead of issued
  bool pdl = true;            // programmatic dependent launches (NLINV_PDL=0 turns them off)
  bool std_fov = false;       // fov = N/4: the passes specialised for it (SizeKernels::row_std, col_std) apply
  bool tc = false;            // radix-16 DFT stages on the tensor cores (params.tensor_dft)
  void* tcB = nullptr;        // their B tiles (workspace)
  double last_alpha = 0.0;    // alpha_n of the last Newton step
  float2* ckpt = nullptr;     // non-null: q_reconstruct writes x_0 .. x_N here (nlinv_reconstruct_checkpoints)
  void* vjp_base = nullptr;   // scratch of nlinv_reconstruct_vjp (allocated on first use)
  std::string err;
};

namespace {

}  // namespace

// Records the message returned by nlinv_last_error(NULL) (used by the calls that take no context).
void nlv_set_global_error(const std::string& msg) { g_create_error = msg; }

namespace {

nlinv_status fail(nlinv_ctx* c, nlinv_status s, const std::string& msg) {
  if (c) c->err = msg; else g_create_error = msg;
  return s;
}

nlinv_status cuda_fail(nlinv_ctx* c, cudaError_t e, const char* where) {
  return fail(c, NLINV_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define NLV_TRY(call, where)                           \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
  } while (0)

KArgs base_args(const nlinv_ctx* c) {
  KArgs a{};
  a.N = c->N;
  a.J = c->J;
  a.f = c->f;
  a.Wc = c->Wc;
  a.wtab = c->wtab;
  a.twA = c->twA;
  a.twB = c->twB;
  a.partials = c->partials;
  a.sc = c->sc;
  a.reduce = nlv::RED_NONE;
  a.tcB = c->tcB;
  return a;
}

nlv::RowGrid row_geom(const nlinv_ctx* c, bool with_rho) {
  if (c->batch_lanes > 0) {           // batch frames: equal block shapes for every frame of a grid side
    nlv::RowGrid g{};
    const int rows = c->J * c->N;
    g.lanes = std::min(c->batch_lanes, rows);
    g.rows_per_cta = g.lanes;
    g.blocks = (rows + g.lanes - 1) / g.lanes;
    g.rho_per_cta = with_rho ? (int)((c->plane + g.blocks - 1) / g.blocks) : 0;
    return g;
  }
  nlv::RowGrid g = nlv::row_grid(c->k, c->J * c->N, with_rho ? c->plane : 0, c->sms, c->row_ctas_per_sm);
  // tensor-core passes: whole warps (every lane of a warp takes part in tcgen05.ld), the extra lanes idle
  if (c->tc)
    while ((g.lanes * c->k->tl) % 32 != 0) ++g.lanes;
  return g;
}

int col_blocks(const nlinv_ctx* c) {
  const int C = c->k->col_lanes;
  return c->J * ((c->Wc + C - 1) / C);
}

// Launches with programmatic stream serialisation (see pdl_enter in kernels.cuh): the next pass is scheduled while
// the current one drains (about 1% per frame on the 384 x 384, 10-coil series).  Every kernel launched here must
// call nlv::pdl_enter() before its first global memory access.
cudaError_t launch(nlinv_ctx* c, const void* fn, int grid, int block, size_t smem, void** args) {
  c->launches++;
  if (c->rec) {                       // every pass takes one KArgs
    c->rec->push_back({fn, grid, block, smem, *(const KArgs*)args[0]});
    return cudaSuccess;
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = c->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = c->pdl ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

cudaError_t row(nlinv_ctx* c, int mode, KArgs a) {
  const bool rho = (mode == nlv::ROW_FFT_W_ADJ || mode == nlv::ROW_FFT_W_NORMAL || mode == nlv::ROW_FFT_W_RHS);
  const nlv::RowGrid g = row_geom(c, rho);
  a.nrows = c->J * c->N;
  a.rows_per_cta = g.rows_per_cta;
  a.rho_per_cta = g.rho_per_cta;
  void* args[] = {&a};
  if (c->tc) {
    const void* fn = (c->std_fov && c->k->row_tc_std[mode]) ? c->k->row_tc_std[mode] : c->k->row_tc[mode];
    return launch(c, fn, g.blocks, g.lanes * c->k->tl, c->k->row_smem_tc(mode, g.lanes), args);
  }
  const void* fn = (c->std_fov && c->k->row_std[mode]) ? c->k->row_std[mode] : c->k->row[mode];
  return launch(c, fn, g.blocks, g.lanes * c->k->tl, c->k->row_smem(mode, g.lanes), args);
}

cudaError_t col(nlinv_ctx* c, int mode, KArgs a) {
  a.nrows = c->J;
  void* args[] = {&a};
  if (c->tc) {
    const void* fn = (c->std_fov && c->k->col_tc_std[mode]) ? c->k->col_tc_std[mode] : c->k->col_tc[mode];
    return launch(c, fn, col_blocks(c), c->k->col_threads, c->k->col_smem_tc(mode, c->Wc), args);
  }
  const void* fn = (c->std_fov && c->k->col_std[mode]) ? c->k->col_std[mode] : c->k->col[mode];
  return launch(c, fn, col_blocks(c), c->k->col_threads, c->k->col_smem(mode, c->Wc), args);
}

// c_j = W^-1 chat_j on Omega, for the coil planes of x (1+J planes).
cudaError_t q_coils(nlinv_ctx* c, const float2* x) {
  KArgs a = base_args(c);
  a.src = x + c->plane;
  a.dst = c->T;
  cudaError_t e = row(c, nlv::ROW_W_IFFT, a);
  if (e != cudaSuccess) return e;
  a = base_args(c);
  a.src = c->T;
  a.dst = c->coil;
  return col(c, nlv::COL_IFFT_C, a);
}

// T <- FFT_col(M rho c_j) for rho = plane 0 of x (coil maps already in c->coil)
cudaError_t q_prod(nlinv_ctx* c, const float2* rho) {
  KArgs a = base_args(c);
  a.rho = rho;
  a.coil = c->coil;
  a.dst = c->T;
  return col(c, nlv::COL_PROD_FFT, a);
}

// T <- FFT_col(M (drho c_j + rho W^-1 dchat_j)) for direction d and linearisation point x
cudaError_t q_dir(nlinv_ctx* c, const float2* x, const float2* d) {
  KArgs a = base_args(c);
  a.src = d + c->plane;
  a.dst = c->T;
  cudaError_t e = row(c, nlv::ROW_W_IFFT, a);
  if (e != cudaSuccess) return e;
  a = base_args(c);
  a.src = c->T;
  a.dst = c->T;
  a.rho = x;
  a.drho = d;
  a.coil = c->coil;
  return col(c, nlv::COL_IFFT_PROD_FFT, a);
}

// T <- FFT_col(conj(rho) z_j), zsum_j <- conj(c_j) z_j, with z_j = M FFT^-1_col(T).  in_cg: a launch of the CG
// iteration (skipped once the solve has stopped).
cudaError_t q_adj_col(nlinv_ctx* c, const float2* x, bool in_cg = false) {
  KArgs a = base_args(c);
  a.cgskip = in_cg ? nlv::kCgSkipEarly : 0;
  a.src = c->T;
  a.dst = c->T;
  a.rho = x;
  a.coil = c->coil;
  a.zsum = c->zsum;
  return col(c, nlv::COL_IFFT_ADJ_FFT, a);
}

// Blocks of the CG step, i.e. the |r|^2 partials the next iteration's first pass adds: one per SM for the bulk-copy
// form of single frames, the vector grid for batch frames.
int cg_blocks(const nlinv_ctx* c) { return c->batch_lanes > 0 ? c->vec_blocks : c->sms; }

// dx += alpha p, r -= alpha q, partials of |r|^2; alpha from the n_pq partials of the normal-operator pass.
// newton / iter: indices of the Newton step and of the CG iteration (recorded if the solve stops here).
cudaError_t q_cg_step(nlinv_ctx* c, int n_pq, int newton, int iter, bool early = true) {
  KArgs a = base_args(c);
  a.cgskip = nlv::kCgSkipAfterWait;
  a.src_early = early ? 1 : 0;
  a.slot = newton;
  a.iter = iter;
  a.pq_part = c->pq_part;
  a.n_pq = n_pq;
  a.rr_part = c->rr_part;
  a.p = c->p;
  a.q = c->q;
  a.r = c->r;
  a.dx = c->dx;
  a.n2 = c->vec / 2;
  void* args[] = {&a};
  if (c->batch_lanes > 0)     // batch frames: the register-staged form, which the batched kernel runs
    return launch(c, cg_step_fn(), c->vec_blocks, kVecThreads, 0, args);
  return launch(c, (const void*)cg_step_bulk, cg_blocks(c), kBulkThreads, kBulkSmem, args);
}

// x += dx
cudaError_t q_add(nlinv_ctx* c) {
  KArgs a = base_args(c);
  a.dx = c->dx;
  a.dst = c->x;
  a.n2 = c->vec / 2;
  void* args[] = {&a};
  return launch(c, (const void*)add_kernel, c->vec_blocks, kVecThreads, 0, args);
}

// One CG iteration on (DF^H DF + alpha) for linearisation point x.  The direction update p = r + beta p of the
// previous iteration is folded into the passes that first read p (beta = 0 right after the right-hand side).
//   K1 row  beta from the |r|^2 partials of K6 before; p_c = r_c + beta p_c; T = W^-1 p_c (first axis)
//   K2 col  drho = r_rho + beta p_rho; T = FFT_col(M (drho c_j + rho W^-1 p_c))
//   K3 row  PSF;  K4 col  adjoint products;  K5 row  q = DF^H DF p + alpha p, p_rho written, Re<p, q> partials
//   K6      alpha from the K5 partials; dx += alpha p, r -= alpha q, per-block partials of |r|^2
// The steps are separate functions so that nlinv_profile_cg times exactly what a reconstruction launches.
// early: p may be loaded before the dependent-launch wait (false for back-to-back launches of this pass alone,
// where each launch would read what the one before writes)
cudaError_t q_cg_k1(nlinv_ctx* c, bool first, bool early = true) {
  KArgs a = base_args(c);
  a.cgskip = nlv::kCgSkipAfterWait;
  a.src = c->p + c->plane;
  a.r = c->r + c->plane;
  a.pupd = 1;
  if (!first) {
    a.rr_part = c->rr_part;
    a.n_rr = cg_blocks(c);
    // p's coil planes were written by this pass one iteration back (before the first iteration, by the
    // right-hand side pass just before it)
    a.src_early = early ? 1 : 0;
  }
  a.dst = c->T;
  return row(c, nlv::ROW_W_IFFT, a);
}

cudaError_t q_cg_k2(nlinv_ctx* c, const float2* x) {
  KArgs a = base_args(c);
  a.cgskip = nlv::kCgSkipEarly;
  a.src = c->T;
  a.dst = c->T;
  a.rho = x;
  a.drho = c->p;
  a.r = c->r;
  a.pupd = 1;
  a.coil = c->coil;
  return col(c, nlv::COL_IFFT_PROD_FFT, a);
}

cudaError_t q_cg_k3(nlinv_ctx* c) {
  KArgs a = base_args(c);
  a.cgskip = nlv::kCgSkipEarly;
  a.src = c->T;
  a.dst = c->T;
  a.mask = c->mask;
  return row(c, nlv::ROW_PSF, a);
}

cudaError_t q_cg_k5(nlinv_ctx* c, float alpha) {
  KArgs a = base_args(c);
  a.cgskip = nlv::kCgSkipEarly;
  a.src = c->T;
  a.dst = c->q;
  a.p = c->p;
  a.r = c->r;
  a.pupd = 1;
  a.zsum = c->zsum;
  a.alpha = alpha;
  a.pq_part = c->pq_part;
  return row(c, nlv::ROW_FFT_W_NORMAL, a);
}

cudaError_t q_cg_iter(nlinv_ctx* c, const float2* x, float alpha, int newton, int iter) {
  cudaError_t e;
  if ((e = q_cg_k1(c, iter == 0)) != cudaSuccess) return e;
  if ((e = q_cg_k2(c, x)) != cudaSuccess) return e;
  if ((e = q_cg_k3(c)) != cudaSuccess) return e;
  if ((e = q_adj_col(c, x, true)) != cudaSuccess) return e;
  if ((e = q_cg_k5(c, alpha)) != cudaSuccess) return e;
  return q_cg_step(c, row_geom(c, true).blocks, newton, iter);
}

// Coil maps of c->x and the Newton residual r0 = y - F x with |r0| into resid[slot].
cudaError_t q_residual(nlinv_ctx* c, int slot) {
  cudaError_t e = q_coils(c, c->x);
  if (e != cudaSuccess) return e;
  if ((e = q_prod(c, c->x)) != cudaSuccess) return e;
  KArgs a = base_args(c);
  a.src = c->T;
  a.dst = c->r0;
  a.y = c->y;
  a.mask = c->mask;
  a.reduce = nlv::RED_RESID;
  a.slot = slot;
  return row(c, nlv::ROW_FFT_RESID, a);
}

// out = a X + b Y over one unknown-space vector ((1+J) planes) or, with planes = J, one data array.
cudaError_t q_axpby(nlinv_ctx* c, float2* out, float a, const float2* X, float b, const float2* Y, long planes) {
  KArgs k = base_args(c);
  k.src = X;
  k.q = Y;
  k.dst = out;
  k.alpha = a;
  k.coef = b;
  k.n2 = planes * c->plane / 2;
  void* args[] = {&k};
  return launch(c, (const void*)axpby_kernel, c->vec_blocks, kVecThreads, 0, args);
}

// out = DF_z d (J data planes) at the linearisation point z.
cudaError_t q_derivative_to(nlinv_ctx* c, const float2* z, const float2* d, const uint8_t* mask, float2* out) {
  cudaError_t e = q_coils(c, z);
  if (e == cudaSuccess) e = q_dir(c, z, d);
  if (e != cudaSuccess) return e;
  KArgs a = base_args(c);
  a.src = c->T;
  a.dst = out;
  a.mask = mask;
  return row(c, nlv::ROW_FFT_P_OUT, a);
}

// out = DF_z^H r (one unknown-space vector) at the linearisation point z.
cudaError_t q_adjoint_to(nlinv_ctx* c, const float2* z, const float2* r, const uint8_t* mask, float2* out) {
  cudaError_t e = q_coils(c, z);
  if (e != cudaSuccess) return e;
  KArgs a = base_args(c);
  a.src = r;
  a.dst = c->T;
  a.mask = mask;
  if ((e = row(c, nlv::ROW_P_IFFT, a)) != cudaSuccess) return e;
  if ((e = q_adj_col(c, z)) != cudaSuccess) return e;
  a = base_args(c);
  a.src = c->T;
  a.dst = out;
  a.zsum = c->zsum;
  return row(c, nlv::ROW_FFT_W_ADJ, a);
}

// The whole reconstruction on the workspace buffers (x, xref, y, mask already in place).
cudaError_t q_reconstruct(nlinv_ctx* c) {
  const nlinv_params& P = c->prm;
  double alpha = P.alpha0;
  cudaError_t e;
  const size_t vb = c->vec * sizeof(float2);
  if (c->ckpt && (e = cudaMemcpyAsync(c->ckpt, c->x, vb, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess) return e;
  for (int n = 0; n < P.newton_steps; ++n) {
    const float al = (float)alpha;
    if ((e = q_residual(c, n)) != cudaSuccess) return e;
    // b = DF^H r0 - alpha (x - xref) -> r = p = b, dx = 0, rr = |b|^2
    KArgs a = base_args(c);
    a.src = c->r0;
    a.dst = c->T;
    a.mask = c->mask;
    if ((e = row(c, nlv::ROW_P_IFFT, a)) != cudaSuccess) return e;
    if ((e = q_adj_col(c, c->x)) != cudaSuccess) return e;
    a = base_args(c);
    a.src = c->T;
    a.zsum = c->zsum;
    a.x = c->x;
    a.xref = c->xref;
    a.r = c->r;
    a.pout = c->p;
    a.dx = c->dx;
    a.alpha = al;
    a.reduce = nlv::RED_RR_INIT;
    a.slot = n;
    if ((e = row(c, nlv::ROW_FFT_W_RHS, a)) != cudaSuccess) return e;
    for (int i = 0; i < P.cg_iters; ++i)
      if ((e = q_cg_iter(c, c->x, al, n, i)) != cudaSuccess) return e;
    if ((e = q_add(c)) != cudaSuccess) return e;
    if (c->ckpt &&
        (e = cudaMemcpyAsync(c->ckpt + (size_t)(n + 1) * c->vec, c->x, vb, cudaMemcpyDeviceToDevice, c->stream)) !=
            cudaSuccess)
      return e;
    c->last_alpha = alpha;
    alpha = std::max(alpha * P.alpha_q, P.alpha_min);
  }
  return q_residual(c, P.newton_steps);
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

nlinv_status check_dev(nlinv_ctx* c, const void* p, const char* name) {
  if (!p) return fail(c, NLINV_EINVAL, std::string(name) + " is NULL");
  if (!is_device_ptr(p)) return fail(c, NLINV_EINVAL, std::string(name) + " must be a device pointer");
  return NLINV_OK;
}

nlinv_status validate(const nlinv_params* p, std::string* why) {
  if (!p) { *why = "params is NULL"; return NLINV_EINVAL; }
  if (!nlinv_supported_size(p->n)) { *why = "grid side n=" + std::to_string(p->n) + " has no compiled transform"; return NLINV_EINVAL; }
  if (p->ncoils < 1 || p->ncoils > 64) { *why = "ncoils must be in 1..64"; return NLINV_EINVAL; }
  if (p->newton_steps < 1 || p->newton_steps > nlv::kMaxNewton) { *why = "newton_steps must be in 1..64"; return NLINV_EINVAL; }
  if (p->cg_iters < 0 || p->cg_iters > 100000) { *why = "cg_iters must be in 0..100000"; return NLINV_EINVAL; }
  if (!(p->alpha0 > 0) || !std::isfinite(p->alpha0)) { *why = "alpha0 must be positive"; return NLINV_EINVAL; }
  if (!(p->alpha_q > 0 && p->alpha_q <= 1)) { *why = "alpha_q must be in (0, 1]"; return NLINV_EINVAL; }
  if (!(p->alpha_min >= 0) || !std::isfinite(p->alpha_min)) { *why = "alpha_min must be >= 0"; return NLINV_EINVAL; }
  if (!(p->sobolev_a >= 0) || !std::isfinite(p->sobolev_a)) { *why = "sobolev_a must be >= 0"; return NLINV_EINVAL; }
  if (!(p->sobolev_l >= 0) || !std::isfinite(p->sobolev_l)) { *why = "sobolev_l must be >= 0"; return NLINV_EINVAL; }
  if (p->fov < 1 || p->fov > p->n / 2) { *why = "fov must be in 1..n/2"; return NLINV_EINVAL; }
  if (p->tensor_dft != 0 && p->tensor_dft != 1) { *why = "tensor_dft must be 0 or 1"; return NLINV_EINVAL; }
  if (p->tensor_dft && !nlv::find_size(p->n)->row_tc[0]) {
    *why = "tensor-core DFT stages are compiled for n = 256 and 512 only";
    return NLINV_EINVAL;
  }
  return NLINV_OK;
}

nlinv_status finish_call(nlinv_ctx* c, cudaError_t e, const char* where) {
  if (e != cudaSuccess) return cuda_fail(c, e, where);
  return NLINV_OK;
}

}  // namespace

// ---------------------------------------------------------------------------------------------- C-ABI ----
extern "C" {

int nlinv_supported_size(int n) { return nlv::find_size(n) != nullptr ? 1 : 0; }

nlinv_status nlinv_default_params(nlinv_params* p, int n, int ncoils) {
  if (!p) return NLINV_EINVAL;
  std::memset(p, 0, sizeof(*p));
  p->n = n;
  p->ncoils = ncoils;
  p->newton_steps = 7;
  p->cg_iters = 30;
  p->alpha0 = 1.0;
  p->alpha_q = 0.5;
  p->alpha_min = 0.0;
  p->sobolev_a = 220.0;
  p->sobolev_l = 32.0;
  p->fov = n / 4;
  p->use_graph = 1;
  p->tensor_dft = 0;
  return NLINV_OK;
}

}  // extern "C"

namespace {

// Twiddle tables of the context's split: twA[k2*N1 + a] = exp(-2 pi i a k2 / N) (a < N1, k2 < N2), twB likewise
// for (N2, N1).  Synchronous.
cudaError_t upload_twiddles(nlinv_ctx* c) {
  const int N = c->N, N1 = c->k->N1, N2 = c->k->N2;
  std::vector<float2> ta(N), tb(N);
  auto tw = [N](long m) {
    m %= N;
    const double t = 2.0 * 3.14159265358979323846 * (double)m / (double)N;
    return make_float2((float)std::cos(t), (float)-std::sin(t));
  };
  for (int k2 = 0; k2 < N2; ++k2)
    for (int a = 0; a < N1; ++a) ta[k2 * N1 + a] = tw((long)a * k2);
  for (int k2 = 0; k2 < N1; ++k2)
    for (int a = 0; a < N2; ++a) tb[k2 * N2 + a] = tw((long)a * k2);
  cudaError_t e = cudaMemcpy(c->twA, ta.data(), N * sizeof(float2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->twB, tb.data(), N * sizeof(float2), cudaMemcpyHostToDevice);
  return e;
}

// Raises the dynamic shared-memory limit of every single-frame pass of table k for the context's shapes; false
// when one of them needs more than the device allows.
bool allow_passes(nlinv_ctx* c, const SizeKernels* k) {
  int smem_optin = 0;
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  const SizeKernels* saved = c->k;
  c->k = k;
  const int lanes = std::max(row_geom(c, false).lanes, row_geom(c, true).lanes);
  c->k = saved;
  auto allow = [&](const void* fn, size_t need) {
    if (!fn) return true;
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) { cudaGetLastError(); return false; }
    const int dyn_max = smem_optin - (int)fa.sharedSizeBytes;
    if ((size_t)dyn_max < need) return false;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return true;
  };
  bool ok = true;
  for (int m = 0; m < nlv::NUM_ROW_MODES && ok; ++m)
    ok = allow(k->row[m], k->row_smem(m, lanes)) && allow(k->row_std[m], k->row_smem(m, lanes));
  for (int m = 0; m < nlv::NUM_COL_MODES && ok; ++m)
    ok = allow(k->col[m], k->col_smem(m, c->Wc)) && allow(k->col_std[m], k->col_smem(m, c->Wc));
  return ok;
}

// Switches the context to the kernel table k (a tuning variant of its side): false, and no change, when its passes
// do not fit; rewrites the twiddle tables when the split differs.  Drops the captured graph.
bool use_variant(nlinv_ctx* c, const SizeKernels* k) {
  if (k == c->k) return true;
  if (!allow_passes(c, k)) return false;
  const bool resplit = k->N1 != c->k->N1;
  c->k = k;
  if (resplit && upload_twiddles(c) != cudaSuccess) return false;
  if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
  return true;
}

// Context set-up shared by nlinv_create and the frames of a batch (batch_lanes > 0: fixed row-pass block shape).
nlinv_status create_ctx(const nlinv_params* params, void* stream, int batch_lanes, nlinv_ctx** out) {
  nlinv_ctx* c = nullptr;
  if (!out) return fail(nullptr, NLINV_EINVAL, "out is NULL");
  *out = nullptr;
  std::string why;
  if (validate(params, &why) != NLINV_OK) return fail(nullptr, NLINV_EINVAL, why);
  c = new (std::nothrow) nlinv_ctx();
  if (!c) return fail(nullptr, NLINV_ENOMEM, "host allocation failed");
  c->prm = *params;
  c->N = params->n;
  c->J = params->ncoils;
  c->f = params->fov;
  c->Wc = 2 * params->fov;
  c->std_fov = 4 * params->fov == params->n;
  c->tc = params->tensor_dft != 0;
  c->plane = (long)c->N * c->N;
  c->vec = (long)(1 + c->J) * c->plane;
  c->k = nlv::find_size(c->N);
  c->batch_lanes = batch_lanes;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) { g_create_error = std::string("cudaGetDevice: ") + cudaGetErrorString(e); delete c; return NLINV_ECUDA; }
  if (stream) {
    c->stream = (cudaStream_t)stream;
  } else {
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { g_create_error = std::string("cudaStreamCreate: ") + cudaGetErrorString(e); delete c; return NLINV_ECUDA; }
    c->own_stream = true;
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  if (const char* v = std::getenv("NLINV_PDL")) c->pdl = std::strcmp(v, "0") != 0;
  c->sms = std::max(1, sms);
  c->vec_blocks = c->sms * NLV_VEC_BLOCKS_PER_SM;
  if (batch_lanes > 0)   // a frame of a batch: vector passes get blocks in proportion to its size
    c->vec_blocks = (int)std::min<long>(c->vec_blocks, std::max<long>(1, c->vec / 2 / (kVecThreads * 8)));

  // dynamic shared memory above the 48 KB default, within the device's opt-in limit
  int smem_optin = 0;
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  // (the limit is raised to the device maximum so that contexts with different fov can share the kernels)
  std::string smem_err;
  auto allow = [&](const void* fn, size_t need) {
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) { smem_err = "cudaFuncGetAttributes failed"; return; }
    const int dyn_max = smem_optin - (int)fa.sharedSizeBytes;
    if ((size_t)dyn_max < need) {
      smem_err = "a pass needs " + std::to_string(need) + " bytes of dynamic shared memory, the device allows " +
                 std::to_string(dyn_max);
      return;
    }
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max) != cudaSuccess)
      smem_err = "cudaFuncSetAttribute failed";
  };
  const int lanes_max = std::max(row_geom(c, false).lanes, row_geom(c, true).lanes);
  for (int m = 0; m < nlv::NUM_ROW_MODES && smem_err.empty(); ++m) {
    allow(c->k->row[m], c->k->row_smem(m, lanes_max));
    if (smem_err.empty()) allow(c->k->row_batch[m], c->k->row_smem(m, lanes_max));
    if (smem_err.empty() && c->k->row_std[m]) allow(c->k->row_std[m], c->k->row_smem(m, lanes_max));
    if (smem_err.empty() && c->k->row_std_batch[m]) allow(c->k->row_std_batch[m], c->k->row_smem(m, lanes_max));
  }
  for (int m = 0; m < nlv::NUM_COL_MODES && smem_err.empty(); ++m) {
    allow(c->k->col[m], c->k->col_smem(m, c->Wc));
    if (smem_err.empty()) allow(c->k->col_batch[m], c->k->col_smem(m, c->Wc));
    if (smem_err.empty() && c->k->col_std[m]) allow(c->k->col_std[m], c->k->col_smem(m, c->Wc));
    if (smem_err.empty() && c->k->col_std_batch[m]) allow(c->k->col_std_batch[m], c->k->col_smem(m, c->Wc));
  }
  if (smem_err.empty()) allow((const void*)cg_step_bulk, kBulkSmem);
  if (c->tc) {
    for (int m = 0; m < nlv::NUM_ROW_MODES && smem_err.empty(); ++m) {
      if (c->k->row_tc[m]) allow(c->k->row_tc[m], c->k->row_smem_tc(m, lanes_max));
      if (smem_err.empty() && c->k->row_tc_std[m]) allow(c->k->row_tc_std[m], c->k->row_smem_tc(m, lanes_max));
    }
    for (int m = 0; m < nlv::NUM_COL_MODES && smem_err.empty(); ++m) {
      if (c->k->col_tc[m]) allow(c->k->col_tc[m], c->k->col_smem_tc(m, c->Wc));
      if (smem_err.empty() && c->k->col_tc_std[m]) allow(c->k->col_tc_std[m], c->k->col_smem_tc(m, c->Wc));
    }
  }
  if (!smem_err.empty()) {
    cudaGetLastError();
    g_create_error = smem_err;
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return NLINV_EINVAL;
  }

  // workspace layout
  const size_t cplx = sizeof(float2);
  const size_t vecb = align_up(c->vec * cplx, 256), datab = align_up((size_t)c->J * c->plane * cplx, 256);
  const size_t Tb = align_up((size_t)c->J * c->N * c->Wc * cplx, 256);
  const size_t cb = align_up((size_t)c->J * c->Wc * c->Wc * cplx, 256);
  const size_t twb = align_up((size_t)c->N * cplx, 256);
  const size_t wb = align_up((size_t)c->plane * sizeof(float), 256);
  const size_t maskb = align_up((size_t)c->plane, 256);
  // partials sized for the largest vector grid that nlinv_autotune tries
  const int max_blocks = std::max(row_geom(c, true).blocks, std::max(c->vec_blocks, c->sms * kTuneVecMax));
  const size_t partb = align_up((size_t)max_blocks * sizeof(double), 256);
  const size_t scb = align_up(sizeof(Scalars), 256);
  const size_t tcb = c->tc ? align_up(nlv::kTcBBytes, 256) : 0;
  const size_t total = 6 * vecb + 2 * datab + Tb + 2 * cb + 2 * twb + wb + maskb + 3 * partb + scb + tcb;
  // NLINV_TEST_FAIL_ALLOC=1 (tests only): the workspace allocation reports out-of-memory without trying, so that
  // the ENOMEM path can be exercised without exhausting a GPU.
  const char* fail_alloc = std::getenv("NLINV_TEST_FAIL_ALLOC");
  e = (fail_alloc && std::strcmp(fail_alloc, "1") == 0) ? cudaErrorMemoryAllocation : cudaMalloc(&c->base, total);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->base = nullptr;
    g_create_error = "cudaMalloc of " + std::to_string(total) + " bytes failed: " + cudaGetErrorString(e);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return NLINV_ENOMEM;
  }
  char* b = (char*)c->base;
  auto take = [&](size_t n) { char* r = b; b += n; return r; };
  c->x = (float2*)take(vecb);
  c->xref = (float2*)take(vecb);
  c->r = (float2*)take(vecb);
  c->p = (float2*)take(vecb);
  c->q = (float2*)take(vecb);
  c->dx = (float2*)take(vecb);
  c->y = (float2*)take(datab);
  c->r0 = (float2*)take(datab);
  c->T = (float2*)take(Tb);
  c->coil = (float2*)take(cb);
  c->zsum = (float2*)take(cb);
  c->twA = (float2*)take(twb);
  c->twB = (float2*)take(twb);
  c->wtab = (float*)take(wb);
  c->mask = (uint8_t*)take(maskb);
  c->partials = (double*)take(partb);
  c->pq_part = (double*)take(partb);
  c->rr_part = (double*)take(partb);
  c->sc = (Scalars*)take(scb);
  if (c->tc) c->tcB = take(tcb);

  const int N = c->N;
  // Sobolev weight w(k) = (1 + a |k|^2)^(-l/2), |k|^2 = (g1^2 + g2^2) / N^2 with signed natural-order indices
  std::vector<float> wt((size_t)c->plane);
  for (int k1 = 0; k1 < N; ++k1)
    for (int k2 = 0; k2 < N; ++k2) {
      const double g1 = k1 < N / 2 ? k1 : k1 - N, g2 = k2 < N / 2 ? k2 : k2 - N;
      const double kk = (g1 * g1 + g2 * g2) / ((double)N * N);
      wt[(size_t)k1 * N + k2] = (float)std::pow(1.0 + params->sobolev_a * kk, -0.5 * params->sobolev_l);
    }
  e = cudaMemset(c->base, 0, total);
  if (e == cudaSuccess) e = upload_twiddles(c);
  if (e == cudaSuccess) e = cudaMemcpy(c->wtab, wt.data(), wt.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && c->tc) {
    std::vector<uint16_t> bt(nlv::kTcBBytes / 2);
    nlv::host_tc_btables(bt.data());
    e = cudaMemcpy(c->tcB, bt.data(), nlv::kTcBBytes, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    g_create_error = std::string("context set-up: ") + cudaGetErrorString(e);
    cudaFree(c->base);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return NLINV_ECUDA;
  }
  *out = c;
  return NLINV_OK;
}

}  // namespace

extern "C" {

nlinv_status nlinv_create(const nlinv_params* params, void* stream, nlinv_ctx** out) {
  return create_ctx(params, stream, 0, out);
}

nlinv_status nlinv_destroy(nlinv_ctx* c) {
  if (!c) return NLINV_OK;
  cudaStreamSynchronize(c->stream);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  cudaFree(c->base);
  if (c->vjp_base) cudaFree(c->vjp_base);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
  return NLINV_OK;
}

nlinv_status nlinv_forward(nlinv_ctx* c, const nlinv_c32* x, const uint8_t* mask, nlinv_c32* y_out) {
  if (!c) return NLINV_EINVAL;
  nlinv_status s;
  if ((s = check_dev(c, x, "x")) || (s = check_dev(c, mask, "mask")) || (s = check_dev(c, y_out, "y_out"))) return s;
  c->launches = 0;
  const float2* xv = (const float2*)x;
  cudaError_t e = q_coils(c, xv);
  if (e == cudaSuccess) e = q_prod(c, xv);
  if (e == cudaSuccess) {
    KArgs a = base_args(c);
    a.src = c->T;
    a.dst = (float2*)y_out;
    a.mask = mask;
    e = row(c, nlv::ROW_FFT_P_OUT, a);
  }
  return finish_call(c, e, "nlinv_forward");
}

nlinv_status nlinv_derivative(nlinv_ctx* c, const nlinv_c32* x, const uint8_t* mask, const nlinv_c32* dx,
                              nlinv_c32* out) {
  if (!c) return NLINV_EINVAL;
  nlinv_status s;
  if ((s = check_dev(c, x, "x")) || (s = check_dev(c, mask, "mask")) || (s = check_dev(c, dx, "dx")) ||
      (s = check_dev(c, out, "out")))
    return s;
  c->launches = 0;
  const cudaError_t e = q_derivative_to(c, (const float2*)x, (const float2*)dx, mask, (float2*)out);
  return finish_call(c, e, "nlinv_derivative");
}

nlinv_status nlinv_adjoint(nlinv_ctx* c, const nlinv_c32* x, const uint8_t* mask, const nlinv_c32* r,
                           nlinv_c32* out) {
  if (!c) return NLINV_EINVAL;
  nlinv_status s;
  if ((s = check_dev(c, x, "x")) || (s = check_dev(c, mask, "mask")) || (s = check_dev(c, r, "r")) ||
      (s = check_dev(c, out, "out")))
    return s;
  c->launches = 0;
  const cudaError_t e = q_adjoint_to(c, (const float2*)x, (const float2*)r, mask, (float2*)out);
  return finish_call(c, e, "nlinv_adjoint");
}

nlinv_status nlinv_normal(nlinv_ctx* c, const nlinv_c32* x, const uint8_t* mask, const nlinv_c32* d, double alpha,
                          nlinv_c32* out) {
  if (!c) return NLINV_EINVAL;
  nlinv_status s;
  if ((s = check_dev(c, x, "x")) || (s = check_dev(c, mask, "mask")) || (s = check_dev(c, d, "d")) ||
      (s = check_dev(c, out, "out")))
    return s;
  if (!std::isfinite(alpha)) return fail(c, NLINV_EINVAL, "alpha must be finite");
  c->launches = 0;
  const float2* xv = (const float2*)x;
  cudaError_t e = q_coils(c, xv);
  if (e == cudaSuccess) e = q_dir(c, xv, (const float2*)d);
  if (e == cudaSuccess) {
    KArgs a = base_args(c);
    a.src = c->T;
    a.dst = c->T;
    a.mask = mask;
    e = row(c, nlv::ROW_PSF, a);
  }
  if (e == cudaSuccess) e = q_adj_col(c, xv);
  if (e == cudaSuccess) {
    KArgs a = base_args(c);
    a.src = c->T;
    a.dst = (float2*)out;
    a.p = (const float2*)d;
    a.zsum = c->zsum;
    a.alpha = (float)alpha;
    a.reduce = nlv::RED_NONE;
    e = row(c, nlv::ROW_FFT_W_NORMAL, a);
  }
  return finish_call(c, e, "nlinv_normal");
}

nlinv_status nlinv_image(nlinv_ctx* c, const nlinv_c32* x, nlinv_c32* image_out) {
  if (!c) return NLINV_EINVAL;
  nlinv_status s;
  if ((s = check_dev(c, x, "x")) || (s = check_dev(c, image_out, "image_out"))) return s;
  c->launches = 0;
  cudaError_t e = q_coils(c, (const float2*)x);
  if (e == cudaSuccess) {
    KArgs a = base_args(c);
    a.rho = (const float2*)x;
    a.coil = c->coil;
    a.dst = (float2*)image_out;
    void* args[] = {&a};
    e = launch(c, (const void*)image_kernel, c->vec_blocks, kVecThreads, 0, args);
  }
  return finish_call(c, e, "nlinv_image");
}

nlinv_status nlinv_simulate(nlinv_ctx* c, const nlinv_c32* rho, const nlinv_c32* coil_img, const uint8_t* mask,
                            nlinv_c32* y_out) {
  if (!c) return NLINV_EINVAL;
  nlinv_status s;
  if ((s = check_dev(c, rho, "rho")) || (s = check_dev(c, coil_img, "coil_img")) ||
      (s = check_dev(c, mask, "mask")) || (s = check_dev(c, y_out, "y_out")))
    return s;
  c->launches = 0;
  KArgs a = base_args(c);
  a.rho = (const float2*)rho;
  a.cimg = (const float2*)coil_img;
  a.dst = c->T;
  cudaError_t e = col(c, nlv::COL_SIM_FFT, a);
  if (e == cudaSuccess) {
    a = base_args(c);
    a.src = c->T;
    a.dst = (float2*)y_out;
    a.mask = mask;
    e = row(c, nlv::ROW_FFT_P_OUT, a);
  }
  return finish_call(c, e, "nlinv_simulate");
}

nlinv_status nlinv_reconstruct(nlinv_ctx* c, const nlinv_c32* y, const uint8_t* mask, const nlinv_c32* x_ref,
                               nlinv_c32* x_inout, double* resid) {
  if (!c) return NLINV_EINVAL;
  if (!y || !mask || !x_inout) return fail(c, NLINV_EINVAL, "y, mask and x_inout must not be NULL");
  const size_t vb = c->vec * sizeof(float2), db = (size_t)c->J * c->plane * sizeof(float2);
  const bool host_x = !is_device_ptr(x_inout);
  NLV_TRY(cudaMemcpyAsync(c->y, y, db, cudaMemcpyDefault, c->stream), "copy y");
  NLV_TRY(cudaMemcpyAsync(c->mask, mask, (size_t)c->plane, cudaMemcpyDefault, c->stream), "copy mask");
  NLV_TRY(cudaMemcpyAsync(c->x, x_inout, vb, cudaMemcpyDefault, c->stream), "copy x");
  NLV_TRY(cudaMemcpyAsync(c->xref, x_ref ? (const void*)x_ref : (const void*)c->x, vb, cudaMemcpyDefault, c->stream),
          "copy x_ref");
  if (c->prm.use_graph) {
    if (!c->graph) {
      cudaGraph_t g = nullptr;
      c->launches = 0;
      NLV_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
      cudaError_t e = q_reconstruct(c);
      cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(c, e != cudaSuccess ? e : e2, "capture reconstruction");
      }
      e = cudaGraphInstantiate(&c->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) { c->graph = nullptr; return cuda_fail(c, e, "instantiate graph"); }
      c->graph_launches = c->launches;
    }
    NLV_TRY(cudaGraphLaunch(c->graph, c->stream), "graph launch");
    c->launches = c->graph_launches;
  } else {
    c->launches = 0;
    NLV_TRY(q_reconstruct(c), "reconstruction");
  }
  c->have_state = true;
  NLV_TRY(cudaMemcpyAsync(x_inout, c->x, vb, cudaMemcpyDefault, c->stream), "copy x out");
  if (resid || host_x) {
    Scalars hs{};
    NLV_TRY(cudaMemcpyAsync(&hs, c->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, c->stream), "read scalars");
    NLV_TRY(cudaStreamSynchronize(c->stream), "synchronize");
    if (resid)
      for (int n = 0; n <= c->prm.newton_steps; ++n) resid[n] = hs.resid[n];
    if (hs.flags & (nlv::kFlagTcTimeout | kFlagCopyTimeout)) {
      int zero = 0;
      cudaMemcpy(&c->sc->flags, &zero, sizeof(int), cudaMemcpyHostToDevice);
      return fail(c, NLINV_ECUDA, "an asynchronous copy or tensor-core stage did not complete within its time limit");
    }
    if (hs.flags & 1) {
      int zero = 0;
      cudaMemcpy(&c->sc->flags, &zero, sizeof(int), cudaMemcpyHostToDevice);
      return fail(c, NLINV_EBREAKDOWN, "CG breakdown: a non-finite |r|^2 or Re<p, A p>");
    }
  }
  return NLINV_OK;
}

nlinv_status nlinv_wait(nlinv_ctx* c, double timeout_s) {
  if (!c) return NLINV_EINVAL;
  cudaEvent_t ev;
  NLV_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event create");
  cudaError_t e = cudaEventRecord(ev, c->stream);
  if (e != cudaSuccess) { cudaEventDestroy(ev); return cuda_fail(c, e, "event record"); }
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    e = cudaEventQuery(ev);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) { cudaEventDestroy(ev); return cuda_fail(c, e, "wait"); }
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (timeout_s >= 0 && el > timeout_s) {
      cudaEventDestroy(ev);
      return fail(c, NLINV_ETIMEOUT, "queued work did not finish within the time limit");
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  cudaEventDestroy(ev);
  int flags = 0;
  NLV_TRY(cudaMemcpy(&flags, &c->sc->flags, sizeof(int), cudaMemcpyDeviceToHost), "read flags");
  if (flags & (nlv::kFlagTcTimeout | kFlagCopyTimeout)) {
    int zero = 0;
    NLV_TRY(cudaMemcpy(&c->sc->flags, &zero, sizeof(int), cudaMemcpyHostToDevice), "clear flags");
    return fail(c, NLINV_ECUDA, "an asynchronous copy or tensor-core stage did not complete within its time limit");
  }
  if (flags & 1) {
    int zero = 0;
    NLV_TRY(cudaMemcpy(&c->sc->flags, &zero, sizeof(int), cudaMemcpyHostToDevice), "clear flags");
    return fail(c, NLINV_EBREAKDOWN, "CG breakdown: a non-finite |r|^2 or Re<p, A p>");
  }
  return NLINV_OK;
}

nlinv_status nlinv_reconstruct_checkpoints(nlinv_ctx* c, const nlinv_c32* y, const uint8_t* mask,
                                           const nlinv_c32* x_ref, nlinv_c32* x_inout, nlinv_c32* ckpt,
                                           double* resid) {
  if (!c) return NLINV_EINVAL;
  nlinv_status s;
  if ((s = check_dev(c, y, "y")) || (s = check_dev(c, mask, "mask")) || (s = check_dev(c, x_inout, "x_inout")) ||
      (s = check_dev(c, ckpt, "ckpt")))
    return s;
  if (x_ref && (s = check_dev(c, x_ref, "x_ref"))) return s;
  const size_t vb = c->vec * sizeof(float2), db = (size_t)c->J * c->plane * sizeof(float2);
  NLV_TRY(cudaMemcpyAsync(c->y, y, db, cudaMemcpyDeviceToDevice, c->stream), "copy y");
  NLV_TRY(cudaMemcpyAsync(c->mask, mask, (size_t)c->plane, cudaMemcpyDeviceToDevice, c->stream), "copy mask");
  NLV_TRY(cudaMemcpyAsync(c->x, x_inout, vb, cudaMemcpyDeviceToDevice, c->stream), "copy x");
  NLV_TRY(cudaMemcpyAsync(c->xref, x_ref ? (const void*)x_ref : (const void*)c->x, vb, cudaMemcpyDeviceToDevice,
                          c->stream), "copy x_ref");
  c->launches = 0;
  c->ckpt = (float2*)ckpt;
  const cudaError_t e = q_reconstruct(c);
  c->ckpt = nullptr;
  NLV_TRY(e, "reconstruction");
  c->have_state = true;
  NLV_TRY(cudaMemcpyAsync(x_inout, c->x, vb, cudaMemcpyDeviceToDevice, c->stream), "copy x out");
  if (resid) {
    Scalars hs{};
    NLV_TRY(cudaMemcpyAsync(&hs, c->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, c->stream), "read scalars");
    NLV_TRY(cudaStreamSynchronize(c->stream), "synchronize");
    for (int n = 0; n <= c->prm.newton_steps; ++n) resid[n] = hs.resid[n];
    if (hs.flags & 1) {
      int zero = 0;
      cudaMemcpy(&c->sc->flags, &zero, sizeof(int), cudaMemcpyHostToDevice);
      return fail(c, NLINV_EBREAKDOWN, "CG breakdown: a non-finite |r|^2 or Re<p, A p>");
    }
  }
  return NLINV_OK;
}

nlinv_status nlinv_reconstruct_vjp(nlinv_ctx* c, const nlinv_c32* y, const uint8_t* mask, const nlinv_c32* ckpt,
                                   const nlinv_c32* grad_x, int tied, nlinv_c32* grad_y, nlinv_c32* grad_x0,
                                   nlinv_c32* grad_xref) {
  if (!c) return NLINV_EINVAL;
  nlinv_status s;
  if ((s = check_dev(c, y, "y")) || (s = check_dev(c, mask, "mask")) || (s = check_dev(c, ckpt, "ckpt")) ||
      (s = check_dev(c, grad_x, "grad_x")) || (s = check_dev(c, grad_y, "grad_y")) ||
      (s = check_dev(c, grad_x0, "grad_x0")))
    return s;
  if (grad_xref && (s = check_dev(c, grad_xref, "grad_xref"))) return s;
  const nlinv_params& P = c->prm;
  const long J = c->J, V = 1 + J;
  const size_t vb = c->vec * sizeof(float2), db = (size_t)J * c->plane * sizeof(float2);
  if (!c->vjp_base) {   // g, dx_n, one adjoint result, dL/dx_ref; s and DF_x u (data arrays)
    cudaError_t e = cudaMalloc(&c->vjp_base, 4 * vb + 2 * db);
    if (e != cudaSuccess) {
      cudaGetLastError();
      c->vjp_base = nullptr;
      return fail(c, NLINV_ENOMEM, "nlinv_reconstruct_vjp: scratch allocation failed");
    }
  }
  float2* g = (float2*)c->vjp_base;
  float2* dxn = g + c->vec;
  float2* tmp = dxn + c->vec;
  float2* gref = tmp + c->vec;
  float2* sres = gref + c->vec;
  float2* v = sres + J * c->plane;
  const float2* X = (const float2*)ckpt;
  c->launches = 0;
  NLV_TRY(cudaMemcpyAsync(c->y, y, db, cudaMemcpyDeviceToDevice, c->stream), "copy y");
  NLV_TRY(cudaMemcpyAsync(c->mask, mask, (size_t)c->plane, cudaMemcpyDeviceToDevice, c->stream), "copy mask");
  NLV_TRY(cudaMemcpyAsync(g, grad_x, vb, cudaMemcpyDeviceToDevice, c->stream), "copy grad_x");
  NLV_TRY(cudaMemsetAsync(grad_y, 0, db, c->stream), "clear grad_y");
  NLV_TRY(cudaMemsetAsync(gref, 0, vb, c->stream), "clear dL/dx_ref");
  std::vector<double> alphas(P.newton_steps);
  double al = P.alpha0;
  for (int n = 0; n < P.newton_steps; ++n) {
    alphas[n] = al;
    al = std::max(al * P.alpha_q, P.alpha_min);
  }
  cudaError_t e = cudaSuccess;
  for (int k = P.newton_steps - 1; k >= 0 && e == cudaSuccess; --k) {
    const float alpha = (float)alphas[k];
    const float2* xk = X + (size_t)k * c->vec;
    e = cudaMemcpyAsync(c->x, xk, vb, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = q_axpby(c, dxn, 1.f, xk + c->vec, -1.f, xk, V);
    // r0 = y - F x_k, then s = r0 - DF_x dx_k (both as "data minus masked transform" row passes)
    if (e == cudaSuccess) e = q_coils(c, c->x);
    if (e == cudaSuccess) e = q_prod(c, c->x);
    if (e == cudaSuccess) {
      KArgs a = base_args(c);
      a.src = c->T; a.dst = c->r0; a.y = c->y; a.mask = c->mask;
      e = row(c, nlv::ROW_FFT_RESID, a);
    }
    if (e == cudaSuccess) e = q_dir(c, c->x, dxn);
    if (e == cudaSuccess) {
      KArgs a = base_args(c);
      a.src = c->T; a.dst = sres; a.y = c->r0; a.mask = c->mask;
      e = row(c, nlv::ROW_FFT_RESID, a);
    }
    // u = (DF^H DF + alpha)^-1 g by the reconstruction's CG (u in c->dx)
    if (e == cudaSuccess) {
      KArgs a = base_args(c);
      a.src = g; a.r = c->r; a.pout = c->p; a.dx = c->dx; a.n2 = c->vec / 2; a.reduce = nlv::RED_RR_INIT;
      a.slot = k;
      void* args[] = {&a};
      e = launch(c, (const void*)cg_init_kernel, c->vec_blocks, kVecThreads, 0, args);
    }
    for (int i = 0; i < P.cg_iters && e == cudaSuccess; ++i) e = q_cg_iter(c, c->x, alpha, k, i);
    // v = DF_x u; dL/dy += v; dL/dx_ref += alpha u
    if (e == cudaSuccess) e = q_dir(c, c->x, c->dx);
    if (e == cudaSuccess) {
      KArgs a = base_args(c);
      a.src = c->T; a.dst = v; a.mask = c->mask;
      e = row(c, nlv::ROW_FFT_P_OUT, a);
    }
    if (e == cudaSuccess) e = q_axpby(c, (float2*)grad_y, 1.f, (const float2*)grad_y, 1.f, v, J);
    if (e == cudaSuccess) e = q_axpby(c, gref, 1.f, gref, alpha, c->dx, V);
    // g <- DF_u^H s - DF_dx^H v
    if (e == cudaSuccess) e = q_adjoint_to(c, c->dx, sres, c->mask, tmp);
    if (e == cudaSuccess) e = q_adjoint_to(c, dxn, v, c->mask, g);
    if (e == cudaSuccess) e = q_axpby(c, g, 1.f, tmp, -1.f, g, V);
  }
  // dL/dx_0 (plus dL/dx_ref when the reference is the start value)
  if (e == cudaSuccess) e = q_axpby(c, (float2*)grad_x0, 1.f, g, tied ? 1.f : 0.f, gref, V);
  if (e == cudaSuccess && grad_xref) e = cudaMemcpyAsync(grad_xref, gref, vb, cudaMemcpyDeviceToDevice, c->stream);
  return finish_call(c, e, "nlinv_reconstruct_vjp");
}

nlinv_status nlinv_profile_cg(nlinv_ctx* c, int reps, double* ms_out) {
  if (!c) return NLINV_EINVAL;
  if (reps < 1 || !ms_out) return fail(c, NLINV_EINVAL, "reps must be >= 1 and ms_out non-NULL");
  if (!c->have_state) return fail(c, NLINV_EINVAL, "run nlinv_reconstruct before nlinv_profile_cg");
  constexpr int K = kProfileKernels;
  // the kernels are timed doing their full work: a solve that stopped at its floor is marked running again
  {
    int flags = 0;
    NLV_TRY(cudaMemcpy(&flags, &c->sc->flags, sizeof(int), cudaMemcpyDeviceToHost), "read flags");
    flags &= ~nlv::kFlagCgStopped;
    NLV_TRY(cudaMemcpy(&c->sc->flags, &flags, sizeof(int), cudaMemcpyHostToDevice), "write flags");
  }
  cudaEvent_t ev[2];
  for (int i = 0; i < 2; ++i) NLV_TRY(cudaEventCreate(&ev[i]), "event create");
  const float al = (float)c->last_alpha;
  // kernel k of the CG iteration, reps launches back to back between two events: its steady-state launch
  // duration (consecutive launches overlap ramp and drain through the dependent launch, as in a graph replay)
  auto one = [&](int k) -> cudaError_t {
    switch (k) {
      case 0: return q_cg_k1(c, false, false);
      case 1: return q_cg_k2(c, c->x);
      case 2: return q_cg_k3(c);
      case 3: return q_adj_col(c, c->x, true);
      case 4: return q_cg_k5(c, al);
      default: return q_cg_step(c, row_geom(c, true).blocks, 0, 0, false);
    }
  };
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < K && e == cudaSuccess; ++k) {
    e = cudaEventRecord(ev[0], c->stream);
    for (int it = 0; it < reps && e == cudaSuccess; ++it) e = one(k);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], c->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    ms_out[k] = ms / reps;
  }
  for (int i = 0; i < 2; ++i) cudaEventDestroy(ev[i]);
  if (e != cudaSuccess) return cuda_fail(c, e, "nlinv_profile_cg");
  return NLINV_OK;
}

long nlinv_last_launch_count(const nlinv_ctx* c) { return c ? c->launches : -1; }

nlinv_status nlinv_cg_stops(nlinv_ctx* c, int* out, int len) {
  if (!c) return NLINV_EINVAL;
  if (!out || len < c->prm.newton_steps) return fail(c, NLINV_EINVAL, "out must hold newton_steps entries");
  if (!c->have_state) return fail(c, NLINV_EINVAL, "no reconstruction has run on this context");
  Scalars hs{};
  NLV_TRY(cudaMemcpyAsync(&hs, c->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, c->stream), "read scalars");
  NLV_TRY(cudaStreamSynchronize(c->stream), "synchronize");
  for (int n = 0; n < c->prm.newton_steps; ++n) out[n] = hs.cg_stop[n];
  return NLINV_OK;
}

nlinv_status nlinv_set_shapes(nlinv_ctx* c, const nlinv_tuning* t) {
  if (!c) return NLINV_EINVAL;
  if (!t) return fail(c, NLINV_EINVAL, "t is NULL");
  if (c->batch_lanes > 0) return fail(c, NLINV_EINVAL, "batch frames keep the batch's shapes");
  if (t->vec_blocks_per_sm < 1 || t->vec_blocks_per_sm > kTuneVecMax)
    return fail(c, NLINV_EINVAL, "vec_blocks_per_sm must be in 1..8");
  if (t->row_blocks_per_sm < 1 || t->row_blocks_per_sm > 3) return fail(c, NLINV_EINVAL, "row_blocks_per_sm must be in 1..3");
  const SizeKernels* variants[8];
  const int nvar = nlv::size_variants(c->N, variants, 8);
  const SizeKernels* pick = nullptr;
  for (int v = 0; v < nvar && !pick; ++v)
    if (variants[v]->N1 == t->split_n1 && variants[v]->col_lanes == t->col_strip) pick = variants[v];
  if (!pick) return fail(c, NLINV_EINVAL, "no compiled transform with that split and column strip for this n");
  if (c->tc && pick != variants[0]) return fail(c, NLINV_EINVAL, "the tensor-core passes keep the compiled split and strips");
  const int saved_rc = c->row_ctas_per_sm;
  c->row_ctas_per_sm = t->row_blocks_per_sm;
  if (!use_variant(c, pick) || !allow_passes(c, c->k)) {
    c->row_ctas_per_sm = saved_rc;
    return fail(c, NLINV_EINVAL, "the passes of these shapes do not fit in shared memory");
  }
  c->vec_blocks = c->sms * t->vec_blocks_per_sm;
  c->pdl = t->pdl != 0;
  if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
  return NLINV_OK;
}

nlinv_status nlinv_autotune(nlinv_ctx* c, const nlinv_c32* y, const uint8_t* mask, const nlinv_c32* x0, int reps,
                            nlinv_tuning* out, nlinv_tuning* table, int table_len) {
  if (!c) return NLINV_EINVAL;
  nlinv_status st;
  if ((st = check_dev(c, y, "y")) || (st = check_dev(c, mask, "mask")) || (st = check_dev(c, x0, "x0"))) return st;
  if (reps < 1 || reps > 1000) return fail(c, NLINV_EINVAL, "reps must be in 1..1000");
  if (c->batch_lanes > 0) return fail(c, NLINV_EINVAL, "batch frames are not tuned one by one");
  if (table && table_len < kTuneMaxCandidates)
    return fail(c, NLINV_EINVAL, "table needs " + std::to_string(kTuneMaxCandidates) + " entries");
  struct Key { int dev, n, J, fov, newton, cg, tc; };
  struct Entry { Key k; const SizeKernels* kern; nlinv_tuning t; std::vector<nlinv_tuning> all; };
  static std::mutex mtx;
  static std::vector<Entry> cache;
  const Key key{c->device, c->N, c->J, c->f, c->prm.newton_steps, c->prm.cg_iters, c->tc ? 1 : 0};
  auto same = [&](const Key& a) {
    return a.dev == key.dev && a.n == key.n && a.J == key.J && a.fov == key.fov && a.newton == key.newton &&
           a.cg == key.cg && a.tc == key.tc;
  };
  // the context's launch shapes as one tuning record (ms_per_frame and stage filled by the caller)
  auto shape = [&]() {
    nlinv_tuning t{};
    t.vec_blocks_per_sm = c->vec_blocks / c->sms;
    t.pdl = c->pdl ? 1 : 0;
    t.split_n1 = c->k->N1;
    t.col_strip = c->k->col_lanes;
    t.row_blocks_per_sm = c->row_ctas_per_sm;
    return t;
  };
  auto set_shapes = [&](int vbk, bool pdl, int row_ctas) {
    c->vec_blocks = c->sms * vbk;
    c->pdl = pdl;
    c->row_ctas_per_sm = row_ctas;
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
  };
  {
    std::lock_guard<std::mutex> lk(mtx);
    for (const Entry& e : cache)
      if (same(e.k)) {
        if (!use_variant(c, e.kern)) return fail(c, NLINV_ECUDA, "nlinv_autotune: cached variant does not fit");
        set_shapes(e.t.vec_blocks_per_sm, e.t.pdl != 0, e.t.row_blocks_per_sm);
        if (out) *out = e.t;
        if (table) {
          for (int i = 0; i < table_len; ++i) table[i] = nlinv_tuning{};
          std::copy(e.all.begin(), e.all.end(), table);
        }
        return NLINV_OK;
      }
  }
  // Whole reconstructions of the caller's frame, replayed as graphs (each replay starts from the same start value):
  // only the whole graph shows how neighbouring passes overlap, and an all-zero workspace times differently from
  // data.  Every timed replay starts with a cold L2 (a write of twice its size outside the events), as a frame of a
  // series does after the rest of an application has run.
  const size_t vb = c->vec * sizeof(float2), db = (size_t)c->J * c->plane * sizeof(float2);
  NLV_TRY(cudaMemcpyAsync(c->y, y, db, cudaMemcpyDeviceToDevice, c->stream), "copy y");
  NLV_TRY(cudaMemcpyAsync(c->mask, mask, (size_t)c->plane, cudaMemcpyDeviceToDevice, c->stream), "copy mask");
  int l2 = 0;
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, c->device);
  const size_t flush_bytes = std::max<size_t>(2 * (size_t)l2, 64u << 20);
  void* flush = nullptr;
  if (cudaMalloc(&flush, flush_bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, NLINV_ENOMEM, "nlinv_autotune: L2 flush buffer allocation failed");
  }
  cudaEvent_t ev[2];
  for (int i = 0; i < 2; ++i) {
    cudaError_t ee = cudaEventCreate(&ev[i]);
    if (ee != cudaSuccess) { cudaFree(flush); return cuda_fail(c, ee, "event create"); }
  }
  cudaError_t e = cudaSuccess;
  // ms per frame of the context's current shapes
  auto time_frame = [&]() -> double {
    if (e != cudaSuccess) return 1e30;
    e = cudaMemcpyAsync(c->x, x0, vb, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->xref, x0, vb, cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return 1e30;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return 1e30;
    cudaError_t e1 = q_reconstruct(c);
    cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
    e = e1 != cudaSuccess ? e1 : e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
    if (g) cudaGraphDestroy(g);
    double tot = 0.0;
    for (int r = 0; r <= reps && e == cudaSuccess; ++r) {          // r = 0: warm-up
      e = cudaMemcpyAsync(c->x, x0, vb, cudaMemcpyDeviceToDevice, c->stream);
      if (e == cudaSuccess) e = cudaMemsetAsync(flush, r & 0xff, flush_bytes, c->stream);
      if (e == cudaSuccess) e = cudaEventRecord(ev[0], c->stream);
      if (e == cudaSuccess) e = cudaGraphLaunch(ge, c->stream);
      if (e == cudaSuccess) e = cudaEventRecord(ev[1], c->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
      if (r > 0) tot += ms;
    }
    if (ge) cudaGraphExecDestroy(ge);
    return e == cudaSuccess ? tot / reps : 1e30;
  };
  Entry ent{};
  // Coordinate descent, one launch-shape dimension per stage, each from the best shapes of the stages before:
  // stage 0 the four-step split of the transforms, 1 the column-strip width, 2 the row-pass blocks per SM, 3 the
  // vector-pass blocks per SM with dependent launch off and on.  Within a stage a candidate replaces the incumbent
  // only when it is kTuneMargin faster (closer shapes swap places with small changes of conditions).
  const SizeKernels* variants[8];
  const int nvar = nlv::size_variants(c->N, variants, 8);
  const SizeKernels* base = c->k;
  auto stage = [&](int id, const std::vector<std::function<bool()>>& cands) {
    // cands[0] restores the incumbent; each candidate applies its shapes and returns false if they do not fit
    double inc_ms = -1.0;
    int best = 0;
    double best_ms = 1e30;
    for (size_t i = 0; i < cands.size() && e == cudaSuccess; ++i) {
      if (!cands[i]()) continue;
      nlinv_tuning t = shape();
      t.ms_per_frame = time_frame();
      t.stage = id;
      if (e != cudaSuccess) break;
      ent.all.push_back(t);
      if (i == 0) inc_ms = t.ms_per_frame;
      if (t.ms_per_frame < best_ms) { best_ms = t.ms_per_frame; best = (int)i; }
    }
    if (inc_ms > 0.0 && best_ms > (1.0 - kTuneMargin) * inc_ms) best = 0;
    if (e == cudaSuccess) cands[best]();
  };
  // stage 0: splits (the default table, and the alternative split if the side has one; the tensor-core passes
  // exist for the default split only)
  {
    std::vector<std::function<bool()>> cands{[&] { return use_variant(c, base); }};
    for (int v = 1; v < nvar && !c->tc; ++v)
      if (variants[v]->N1 != base->N1) cands.push_back([&, v] { return use_variant(c, variants[v]); });
    stage(0, cands);
  }
  // stage 1: column strips of the chosen split (variants of the default split only)
  if (c->k->N1 == base->N1 && !c->tc) {
    std::vector<std::function<bool()>> cands{[&] { return use_variant(c, base); }};
    for (int v = 1; v < nvar; ++v)
      if (variants[v]->N1 == base->N1 && variants[v]->col_lanes != base->col_lanes)
        cands.push_back([&, v] { return use_variant(c, variants[v]); });
    stage(1, cands);
  }
  // stage 2: row-pass blocks per SM
  {
    const int inc = c->row_ctas_per_sm;
    std::vector<std::function<bool()>> cands{[&, inc] { set_shapes(c->vec_blocks / c->sms, c->pdl, inc); return true; }};
    for (int rc : {1, 2, 3})
      if (rc != inc)
        cands.push_back([&, rc] { set_shapes(c->vec_blocks / c->sms, c->pdl, rc); return allow_passes(c, c->k); });
    stage(2, cands);
  }
  // stage 3: vector-pass blocks per SM x dependent launch
  {
    const int ivb = c->vec_blocks / c->sms;
    const bool ipdl = c->pdl;
    std::vector<std::function<bool()>> cands{[&, ivb, ipdl] { set_shapes(ivb, ipdl, c->row_ctas_per_sm); return true; }};
    for (int pdl = 0; pdl < 2; ++pdl)
      for (int vbk : {2, 4, kTuneVecMax})
        if (vbk != ivb || (pdl != 0) != ipdl)
          cands.push_back([&, vbk, pdl] { set_shapes(vbk, pdl != 0, c->row_ctas_per_sm); return true; });
    stage(3, cands);
  }
  for (int i = 0; i < 2; ++i) cudaEventDestroy(ev[i]);
  cudaFree(flush);
  int zero = 0;   // the timing runs are not the caller's results: drop any flag they raised
  if (e == cudaSuccess) e = cudaMemcpy(&c->sc->flags, &zero, sizeof(int), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(c, e, "nlinv_autotune");
  ent.k = key;
  ent.kern = c->k;
  ent.t = shape();
  // the chosen shapes' own measurement: the last stage's entry for them
  for (const nlinv_tuning& t : ent.all)
    if (t.vec_blocks_per_sm == ent.t.vec_blocks_per_sm && t.pdl == ent.t.pdl && t.split_n1 == ent.t.split_n1 &&
        t.col_strip == ent.t.col_strip && t.row_blocks_per_sm == ent.t.row_blocks_per_sm)
      ent.t.ms_per_frame = t.ms_per_frame, ent.t.stage = t.stage;
  {
    std::lock_guard<std::mutex> lk(mtx);
    cache.push_back(ent);
  }
  if (out) *out = ent.t;
  if (table) {
    for (int i = 0; i < table_len; ++i) table[i] = nlinv_tuning{};
    std::copy(ent.all.begin(), ent.all.end(), table);
  }
  return NLINV_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------- batches ----
struct nlinv_batch {
  nlinv_params prm{};
  std::vector<nlinv_ctx*> frames;           // per-frame workspaces (they never launch by themselves)
  std::vector<std::vector<int>> groups;     // frame indices per grid side
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<cudaStream_t> gstream;        // branch stream per group (group 0 runs on `stream`)
  cudaEvent_t ev_fork = nullptr;
  std::vector<cudaEvent_t> ev_join;
  void* tables = nullptr;                   // device: per-launch frame arguments and block offsets
  struct Launch {
    int group;
    const void* fn;
    int grid, block;
    size_t smem;
    nlv::BatchArgs args;
  };
  std::vector<Launch> launches;
  cudaGraphExec_t graph = nullptr;
  bool have_state = false;                  // a reconstruction has filled the workspaces
  std::vector<size_t> group_first;          // index in `launches` of each group's first launch
  bool pdl = true;
  bool multi = false;                       // one launch per pass for all sides the multi-side kernels cover
                                            // (NLINV_BATCH_MULTI=1; measured slower, see nlinv_batch_create)
};

namespace {

void batch_free(nlinv_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (size_t g = 1; g < b->gstream.size(); ++g)
    if (b->gstream[g]) cudaStreamDestroy(b->gstream[g]);
  for (cudaEvent_t e : b->ev_join)
    if (e) cudaEventDestroy(e);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->tables) cudaFree(b->tables);
  for (nlinv_ctx* c : b->frames) nlinv_destroy(c);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

// The multi-side kernel (kernels.cuh, "batches of several sides") that runs the single-frame pass fn of side k for
// frames of every side, and its dynamic shared memory; nullptr if fn is not a pass.
const void* multi_kernel(const SizeKernels* k, const void* fn, size_t* smem) {
  const nlv::MultiKernels* mk = nlv::multi_kernels();
  for (int m = 0; m < nlv::NUM_ROW_MODES; ++m) {
    if (fn == k->row[m]) { *smem = mk->row_smem[m]; return mk->row[m]; }
    if (k->row_std[m] && fn == k->row_std[m]) { *smem = mk->row_smem[m]; return mk->row_std[m]; }
  }
  for (int m = 0; m < nlv::NUM_COL_MODES; ++m) {
    if (fn == k->col[m]) { *smem = mk->col_smem[m]; return mk->col[m]; }
    if (k->col_std[m] && fn == k->col_std[m]) { *smem = mk->col_smem[m]; return mk->col_std[m]; }
  }
  *smem = 0;
  if (fn == cg_step_fn()) return (const void*)cg_step_batch;
  if (fn == (const void*)add_kernel) return (const void*)add_batch;
  return nullptr;
}

// The batched kernel that runs the single-frame pass fn for several frames of one side.
const void* batched_kernel(const SizeKernels* k, const void* fn) {
  for (int m = 0; m < nlv::NUM_ROW_MODES; ++m) {
    if (fn == k->row[m]) return k->row_batch[m];
    if (k->row_std[m] && fn == k->row_std[m]) return k->row_std_batch[m];
  }
  for (int m = 0; m < nlv::NUM_COL_MODES; ++m) {
    if (fn == k->col[m]) return k->col_batch[m];
    if (k->col_std[m] && fn == k->col_std[m]) return k->col_std_batch[m];
  }
  if (fn == cg_step_fn()) return (const void*)cg_step_batch;
  if (fn == (const void*)add_kernel) return (const void*)add_batch;
  return nullptr;
}

// One batched launch on stream st (with the batch's dependent-launch setting).
cudaError_t launch_batched(nlinv_batch* b, nlinv_batch::Launch& bl, cudaStream_t st) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(bl.grid);
  cfg.blockDim = dim3(bl.block);
  cfg.dynamicSmemBytes = bl.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = b->pdl ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[] = {&bl.args};
  return cudaLaunchKernelExC(&cfg, bl.fn, args);
}

nlinv_status batch_fail(nlinv_batch* b, nlinv_status st, const std::string& msg) {
  g_create_error = msg;
  batch_free(b);
  return st;
}

}  // namespace

extern "C" {

nlinv_status nlinv_batch_create(const nlinv_params* params, int nframes, const nlinv_frame_desc* frames,
                                void* stream, nlinv_batch** out) {
  if (!out) return fail(nullptr, NLINV_EINVAL, "out is NULL");
  *out = nullptr;
  if (!params || !frames || nframes < 1 || nframes > 4096)
    return fail(nullptr, NLINV_EINVAL, "params, frames and 1 <= nframes <= 4096 are required");
  nlinv_batch* b = new (std::nothrow) nlinv_batch();
  if (!b) return fail(nullptr, NLINV_ENOMEM, "host allocation failed");
  b->prm = *params;
  if (const char* v = std::getenv("NLINV_PDL")) b->pdl = std::strcmp(v, "0") != 0;
  if (const char* v = std::getenv("NLINV_BATCH_MULTI")) b->multi = std::strcmp(v, "0") != 0;
  cudaError_t e = cudaSuccess;
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return batch_fail(b, NLINV_ECUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    b->own_stream = true;
  }
  // one workspace per frame, grouped by grid side
  std::vector<int> sides;
  for (int i = 0; i < nframes; ++i) {
    nlinv_params fp = *params;
    fp.n = frames[i].n;
    fp.ncoils = frames[i].ncoils;
    fp.fov = frames[i].n / 4;
    fp.use_graph = 0;
    fp.tensor_dft = 0;        // batches run the FP32 transforms
    const SizeKernels* k = nlv::find_size(fp.n);
    if (!k) return batch_fail(b, NLINV_EINVAL, "frame " + std::to_string(i) + ": unsupported grid side");
    nlinv_ctx* c = nullptr;
    const nlinv_status st = create_ctx(&fp, b->stream, nlv::kRowMaxThreads / k->tl, &c);
    if (st != NLINV_OK) return batch_fail(b, st, "frame " + std::to_string(i) + ": " + g_create_error);
    b->frames.push_back(c);
    // frames of the sides the multi-side kernels cover form one group (side key 0); other sides one group each
    const int key = (b->multi && nlv::multi_side(fp.n)) ? 0 : fp.n;
    size_t g = 0;
    while (g < sides.size() && sides[g] != key) ++g;
    if (g == sides.size()) {
      sides.push_back(key);
      b->groups.emplace_back();
    }
    b->groups[g].push_back(i);
  }
  int sms = 1, dev = 0, smem_optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  // the launch sequence of every frame, merged launch by launch within each group
  std::vector<std::vector<nlinv_ctx::Rec>> recs(nframes);
  for (int i = 0; i < nframes; ++i) {
    nlinv_ctx* c = b->frames[i];
    c->rec = &recs[i];
    e = q_reconstruct(c);
    c->rec = nullptr;
    if (e != cudaSuccess) return batch_fail(b, NLINV_ECUDA, std::string("recording: ") + cudaGetErrorString(e));
  }
  std::vector<char> host;
  std::vector<size_t> arg_off, first_off;
  for (size_t g = 0; g < b->groups.size(); ++g) {
    const std::vector<int>& fr = b->groups[g];
    const size_t L = recs[fr[0]].size();
    const SizeKernels* k = b->frames[fr[0]]->k;
    for (int i : fr)
      if (recs[i].size() != L) return batch_fail(b, NLINV_EINVAL, "frames of one grid side differ in schedule");
    const bool multi = sides[g] == 0;
    b->group_first.push_back(b->launches.size());
    for (size_t l = 0; l < L; ++l) {
      nlinv_batch::Launch bl{};
      bl.group = (int)g;
      size_t msmem = 0;
      bl.fn = multi ? multi_kernel(k, recs[fr[0]][l].fn, &msmem) : batched_kernel(k, recs[fr[0]][l].fn);
      if (!bl.fn) return batch_fail(b, NLINV_EINVAL, "internal: no batched form of a pass");
      size_t off = (host.size() + 15) / 16 * 16;
      host.resize(off + fr.size() * sizeof(KArgs));
      arg_off.push_back(off);
      std::vector<int> first(fr.size() + 1, 0);
      bl.block = 0;
      for (size_t t = 0; t < fr.size(); ++t) {
        const nlinv_ctx::Rec& r = recs[fr[t]][l];
        size_t ms = 0;
        const void* same = multi ? multi_kernel(b->frames[fr[t]]->k, r.fn, &ms) : batched_kernel(k, r.fn);
        if (same != bl.fn || (!multi && r.block != recs[fr[0]][l].block))
          return batch_fail(b, NLINV_EINVAL, "frames of one group differ in pass shapes");
        std::memcpy(host.data() + off + t * sizeof(KArgs), &r.args, sizeof(KArgs));
        first[t + 1] = first[t] + r.grid;
        bl.smem = multi ? msmem : std::max(bl.smem, r.smem);
        bl.block = std::max(bl.block, r.block);
      }
      if (multi) {   // the multi-side kernels run fixed block shapes
        const nlv::MultiKernels* mk = nlv::multi_kernels();
        bool is_col = false;
        for (int m = 0; m < nlv::NUM_COL_MODES; ++m)
          is_col = is_col || bl.fn == mk->col[m] || (mk->col_std[m] && bl.fn == mk->col_std[m]);
        bool is_row = false;
        for (int m = 0; m < nlv::NUM_ROW_MODES; ++m)
          is_row = is_row || bl.fn == mk->row[m] || (mk->row_std[m] && bl.fn == mk->row_std[m]);
        if (is_row) bl.block = nlv::kRowMaxThreads;
        if (is_col) bl.block = nlv::kMultiColThreads;
      }
      // persistent blocks: as many as are resident at once, each looping over the work items
      cudaFuncAttributes fa{};
      if (cudaFuncGetAttributes(&fa, bl.fn) == cudaSuccess && bl.smem > 0)
        cudaFuncSetAttribute(bl.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin - (int)fa.sharedSizeBytes);
      int occ = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bl.fn, bl.block, bl.smem) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        return batch_fail(b, NLINV_EINVAL, "a batched pass does not fit on a multiprocessor");
      }
      bl.grid = std::min(first.back(), occ * sms);
      off = (host.size() + 15) / 16 * 16;
      host.resize(off + first.size() * sizeof(int));
      std::memcpy(host.data() + off, first.data(), first.size() * sizeof(int));
      first_off.push_back(off);
      bl.args.nframes = (int)fr.size();
      bl.args.total = first.back();
      b->launches.push_back(bl);
    }
  }
  e = cudaMalloc(&b->tables, host.size());
  if (e != cudaSuccess) { cudaGetLastError(); return batch_fail(b, NLINV_ENOMEM, "batch tables: cudaMalloc failed"); }
  e = cudaMemcpy(b->tables, host.data(), host.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return batch_fail(b, NLINV_ECUDA, std::string("batch tables: ") + cudaGetErrorString(e));
  for (size_t l = 0; l < b->launches.size(); ++l) {
    b->launches[l].args.args = (const KArgs*)((char*)b->tables + arg_off[l]);
    b->launches[l].args.first = (const int*)((char*)b->tables + first_off[l]);
  }
  // one graph: the groups as parallel branches
  const size_t G = b->groups.size();
  b->gstream.assign(G, nullptr);
  b->ev_join.assign(G, nullptr);
  b->gstream[0] = b->stream;
  for (size_t g = 1; g < G && e == cudaSuccess; ++g) {
    e = cudaStreamCreateWithFlags(&b->gstream[g], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join[g], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
  if (e != cudaSuccess) return batch_fail(b, NLINV_ECUDA, std::string("batch streams: ") + cudaGetErrorString(e));
  cudaGraph_t graph = nullptr;
  e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) e = cudaEventRecord(b->ev_fork, b->stream);
  for (size_t g = 1; g < G && e == cudaSuccess; ++g) e = cudaStreamWaitEvent(b->gstream[g], b->ev_fork, 0);
  for (size_t l = 0; l < b->launches.size() && e == cudaSuccess; ++l)
    e = launch_batched(b, b->launches[l], b->gstream[b->launches[l].group]);
  for (size_t g = 1; g < G && e == cudaSuccess; ++g) {
    e = cudaEventRecord(b->ev_join[g], b->gstream[g]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev_join[g], 0);
  }
  cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    b->graph = nullptr;
    return batch_fail(b, NLINV_ECUDA, std::string("batch graph: ") + cudaGetErrorString(e));
  }
  *out = b;
  return NLINV_OK;
}

nlinv_status nlinv_reconstruct_batch(nlinv_batch* b, int nframes, const nlinv_frame_desc* frames) {
  if (!b) return NLINV_EINVAL;
  if (!frames || nframes != (int)b->frames.size())
    return fail(nullptr, NLINV_EINVAL, "nframes and the frames must match the batch");
  bool wait = false;
  for (int i = 0; i < nframes; ++i) {
    nlinv_ctx* c = b->frames[i];
    const nlinv_frame_desc& d = frames[i];
    if (d.n != c->N || d.ncoils != c->J) return fail(nullptr, NLINV_EINVAL, "frame " + std::to_string(i) + ": shape differs");
    if (!d.y || !d.mask || !d.x_inout) return fail(nullptr, NLINV_EINVAL, "frame " + std::to_string(i) + ": NULL buffer");
    wait = wait || d.resid || !is_device_ptr(d.x_inout);
  }
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < nframes && e == cudaSuccess; ++i) {
    nlinv_ctx* c = b->frames[i];
    const nlinv_frame_desc& d = frames[i];
    const size_t vb = c->vec * sizeof(float2), db = (size_t)c->J * c->plane * sizeof(float2);
    e = cudaMemcpyAsync(c->y, d.y, db, cudaMemcpyDefault, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->mask, d.mask, (size_t)c->plane, cudaMemcpyDefault, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->x, d.x_inout, vb, cudaMemcpyDefault, b->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->xref, d.x_ref ? (const void*)d.x_ref : (const void*)c->x, vb, cudaMemcpyDefault, b->stream);
  }
  if (e == cudaSuccess) e = cudaGraphLaunch(b->graph, b->stream);
  if (e == cudaSuccess) b->have_state = true;
  for (int i = 0; i < nframes && e == cudaSuccess; ++i) {
    nlinv_ctx* c = b->frames[i];
    e = cudaMemcpyAsync(frames[i].x_inout, c->x, c->vec * sizeof(float2), cudaMemcpyDefault, b->stream);
  }
  if (e != cudaSuccess) return fail(nullptr, NLINV_ECUDA, std::string("nlinv_reconstruct_batch: ") + cudaGetErrorString(e));
  if (!wait) return NLINV_OK;
  std::vector<Scalars> hs(nframes);
  for (int i = 0; i < nframes && e == cudaSuccess; ++i)
    e = cudaMemcpyAsync(&hs[i], b->frames[i]->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return fail(nullptr, NLINV_ECUDA, std::string("nlinv_reconstruct_batch: ") + cudaGetErrorString(e));
  bool broke = false;
  for (int i = 0; i < nframes; ++i) {
    if (frames[i].resid)
      for (int n = 0; n <= b->prm.newton_steps; ++n) frames[i].resid[n] = hs[i].resid[n];
    if (hs[i].flags & 1) {
      broke = true;
      int zero = 0;
      cudaMemcpy(&b->frames[i]->sc->flags, &zero, sizeof(int), cudaMemcpyHostToDevice);
    }
  }
  if (broke) return fail(nullptr, NLINV_EBREAKDOWN, "CG breakdown in at least one frame");
  return NLINV_OK;
}

long nlinv_batch_launch_count(const nlinv_batch* b) { return b ? (long)b->launches.size() : -1; }

nlinv_status nlinv_batch_profile_cg(nlinv_batch* b, int reps, double* ms_out) {
  if (!b) return NLINV_EINVAL;
  if (reps < 1 || !ms_out) return fail(nullptr, NLINV_EINVAL, "reps must be >= 1 and ms_out non-NULL");
  if (!b->have_state) return fail(nullptr, NLINV_EINVAL, "run nlinv_reconstruct_batch before nlinv_batch_profile_cg");
  if (b->prm.cg_iters < 2) return fail(nullptr, NLINV_EINVAL, "the batch's schedule has fewer than two CG iterations");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  // every frame's solve is marked running, so that every kernel does its full work
  for (nlinv_ctx* c : b->frames) {
    int flags = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&flags, &c->sc->flags, sizeof(int), cudaMemcpyDeviceToHost);
    flags &= ~nlv::kFlagCgStopped;
    if (e == cudaSuccess) e = cudaMemcpy(&c->sc->flags, &flags, sizeof(int), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) return fail(nullptr, NLINV_ECUDA, std::string("nlinv_batch_profile_cg: ") + cudaGetErrorString(e));
  // the six launches of the second CG iteration of the first Newton step, in every group: they end at the group's
  // second CG step
  std::vector<size_t> first6;
  for (size_t g = 0; g < b->group_first.size(); ++g) {
    const size_t end = g + 1 < b->group_first.size() ? b->group_first[g + 1] : b->launches.size();
    int seen = 0;
    size_t at = 0;
    for (size_t l = b->group_first[g]; l < end && seen < 2; ++l)
      if (b->launches[l].fn == (const void*)cg_step_batch && ++seen == 2) at = l;
    if (seen < 2 || at < b->group_first[g] + 5) return fail(nullptr, NLINV_EINVAL, "internal: CG launches not found");
    first6.push_back(at - 5);
  }
  cudaEvent_t ev[2];
  for (int i = 0; i < 2; ++i)
    if ((e = cudaEventCreate(&ev[i])) != cudaSuccess)
      return fail(nullptr, NLINV_ECUDA, std::string("event create: ") + cudaGetErrorString(e));
  for (int k = 0; k < kProfileKernels && e == cudaSuccess; ++k) {
    e = cudaEventRecord(ev[0], b->stream);
    for (int it = 0; it < reps && e == cudaSuccess; ++it)
      for (size_t g = 0; g < first6.size() && e == cudaSuccess; ++g)
        e = launch_batched(b, b->launches[first6[g] + k], b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], b->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    ms_out[k] = ms / reps;
  }
  for (int i = 0; i < 2; ++i) cudaEventDestroy(ev[i]);
  if (e != cudaSuccess) return fail(nullptr, NLINV_ECUDA, std::string("nlinv_batch_profile_cg: ") + cudaGetErrorString(e));
  return NLINV_OK;
}

nlinv_status nlinv_batch_destroy(nlinv_batch* b) {
  batch_free(b);
  return NLINV_OK;
}

const char* nlinv_last_error(const nlinv_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

}  // extern "C"
