// Radix-16 DFT stages on the tensor cores (tcgen05.mma, operands in shared memory, FP32 accumulators in TMEM) in
// split-BF16 with three passes: the optional precision path of the transforms (the paper computes in complex
// single precision, Sec. 3.2; these stages trade FP32 butterflies for bf16 products accumulated in FP32).
//
// One call transforms one vector of 16 complex values per thread of the block:  X_k = sum_n x_n W^{nk},
// W = exp(D 2 pi i / 16).  As a real contraction, the interleaved row [Re x_0, Im x_0, Re x_1, ...] (K = 32) times
// the 32 x 32 real matrix B with B[2n + a][2k + b] = ((cos, sin), (-sin, cos))[a][b] of the angle D 2 pi n k / 16
// gives the interleaved row of X (N = 32).  Each value v is split as v = hi + lo with hi = v truncated to bf16
// and lo = bf16(v - hi) (v - hi is exact in FP32), B likewise (on the host, in double); the three products
// hi*Bhi + hi*Blo + lo*Bhi accumulate in FP32 (the lo*Blo term, ~2^-16 relative, is dropped).
//
// Mapping: thread t of the block owns row t & 127 of the A tile of its warpgroup g = t >> 7; one elected thread
// issues, per warpgroup, 2 K-steps x 3 passes of tcgen05.mma.cta_group::1.kind::f16 (M = 128, N = 32, K = 16)
// into TMEM columns [32 g, 32 g + 32); completion arrives on an mbarrier through tcgen05.commit; every warp then
// reads its 32 lanes back with tcgen05.ld.32x32b.x32 -- thread t gets its own row, i.e. its own 16 outputs.
//
// Shared-memory operand layout (no swizzle, K-major): 8 x 16-byte "core matrices" (8 rows of 8 bf16); for a
// tile of R rows x 32 K, core matrix (row group i, K group k) sits at i * 512 + k * 128 bytes, row r of a core
// matrix at r * 16.  Descriptor: leading-dimension offset (between K groups) 128 B, stride-dimension offset
// (between row groups) 512 B; one K-step of 16 elements = 2 K groups = 256 bytes.
#pragma once
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

namespace nlv {

constexpr int kTcTileBytes = 128 * 32 * 2;          // one A tile: 128 rows x 32 bf16
constexpr int kTcBTileBytes = 32 * 32 * 2;          // one B tile: 32 rows (N) x 32 bf16 (K)
constexpr int kTcBBytes = 4 * kTcBTileBytes;        // B tiles: forward hi, forward lo, inverse hi, inverse lo
constexpr int kFlagTcTimeout = 4;                   // Scalars::flags bit: a tensor-core completion wait timed out

// Byte offset of element (row, k) in a no-swizzle K-major tile (see above).
__host__ __device__ constexpr int tc_tile_offset(int row, int k) {
  return (row >> 3) * 512 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// Shared memory the engine needs for a block of `threads` threads: A tiles (hi and lo per warpgroup), the B tiles,
// the mbarrier and the TMEM address slot.
__host__ __device__ constexpr int tc_warpgroups(int threads) { return (threads + 127) / 128; }
__host__ __device__ constexpr size_t tc_smem_bytes(int threads) {
  return (size_t)tc_warpgroups(threads) * 2 * kTcTileBytes + kTcBBytes + 16;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// 64-bit shared-memory matrix descriptor of tcgen05: start address >> 4 (bits 0-13), leading-dimension byte
// offset >> 4 (bits 16-29), stride-dimension byte offset >> 4 (bits 32-45), descriptor version 1 (bits 46-47),
// base offset 0, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: D in F32 (bits 4-5 = 1), A and B bf16 (bits 7-9, 10-12 = 1), both K-major,
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// bf16 pair {lo half = a, hi half = b}, each rounded to nearest even
__device__ __forceinline__ uint32_t pack_bf16_rn(float a, float b) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
  return r;
}

// v = hi + lo for both parts of a complex value: hi = the bf16 truncations packed (re in the low half), lo = the
// bf16 roundings of the exact FP32 remainders.
__device__ __forceinline__ void tc_split(float2 v, uint32_t& hi, uint32_t& lo) {
  const uint32_t ur = __float_as_uint(v.x), ui = __float_as_uint(v.y);
  hi = __byte_perm(ur, ui, 0x7632);
  const float rr = v.x - __uint_as_float(ur & 0xFFFF0000u);
  const float ri = v.y - __uint_as_float(ui & 0xFFFF0000u);
  lo = pack_bf16_rn(rr, ri);
}

struct TcDft {
  static constexpr bool enabled = true;
  unsigned char* a_tiles;     // shared: per warpgroup hi tile then lo tile
  unsigned char* b_tiles;     // shared: forward hi, forward lo, inverse hi, inverse lo
  uint32_t mbar;              // shared address of the completion barrier
  uint32_t tmem;              // TMEM base address of the accumulators
  uint32_t ncols;             // TMEM columns held
  uint32_t phase;             // parity of the next completion
  int* flags;                 // global flags word (kFlagTcTimeout on a timed-out wait), may be null
  bool timed_out;

  // Set-up by every thread of the block, after the block's first global-memory wait: initialises the barrier,
  // stages the B tiles (from a global table of kTcBBytes, written by cp.async: the caller waits for them with its
  // other staged inputs) and allocates TMEM (warp 0).  smem: tc_smem_bytes(blockDim.x) bytes, 16-byte aligned.
  __device__ __forceinline__ void setup(unsigned char* smem, const void* btab, int* flags_) {
    const int G = tc_warpgroups(blockDim.x);
    a_tiles = smem;
    b_tiles = smem + (size_t)G * 2 * kTcTileBytes;
    uint64_t* bar = (uint64_t*)(b_tiles + kTcBBytes);
    uint32_t* slot = (uint32_t*)(bar + 1);
    mbar = smem_u32(bar);
    flags = flags_;
    phase = 0;
    timed_out = false;
    ncols = 32;
    while (ncols < 32u * G) ncols <<= 1;
    for (int i = threadIdx.x; i < kTcBBytes / 16; i += blockDim.x) {
      const unsigned s = smem_u32(b_tiles + 16 * i);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"((const char*)btab + 16 * i) : "memory");
    }
    if (threadIdx.x == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                   "r"(ncols) : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    tmem = *(volatile uint32_t*)slot;
  }

  // Waits (at most about a second of clock cycles) for the completion of the phase `phase` of the barrier.
  __device__ __forceinline__ bool wait_phase() {
    const long long t0 = clock64();
    for (;;) {
      uint32_t ok;
      asm volatile("{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                   "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(ok) : "r"(mbar), "r"(phase) : "memory");
      if (ok) return true;
      if (clock64() - t0 > 2000000000LL) return false;
      __nanosleep(32);
    }
  }

  // X = DFT16_D(v[0..15]) for every thread's vector (threads with !valid pass zeros and ignore the result).
  // Must be called by every thread of the block (it contains barriers).
  template <int D, int E>
  __device__ __forceinline__ void dft16(float2 (&v)[E], bool valid) {
    static_assert(E >= 16, "a thread holds 16 values");
    const int t = threadIdx.x, g = t >> 7, row = t & 127;
    unsigned char* ahi = a_tiles + (size_t)g * 2 * kTcTileBytes;
    unsigned char* alo = ahi + kTcTileBytes;
    // row t: 4 chunks of 8 bf16 (4 complex values) per tile
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      uint32_t h[4], l[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 x = valid ? v[4 * c + q] : make_float2(0.f, 0.f);
        tc_split(x, h[q], l[q]);
      }
      const int off = tc_tile_offset(row, 8 * c);
      *(uint4*)(ahi + off) = make_uint4(h[0], h[1], h[2], h[3]);
      *(uint4*)(alo + off) = make_uint4(l[0], l[1], l[2], l[3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (t == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int G = tc_warpgroups(blockDim.x);
      const unsigned char* bh = b_tiles + (D < 0 ? 0 : 2) * kTcBTileBytes;
      const unsigned char* bl = bh + kTcBTileBytes;
      constexpr uint32_t idesc = tc_idesc(128, 32);
      for (int gg = 0; gg < G; ++gg) {
        const unsigned char* ah = a_tiles + (size_t)gg * 2 * kTcTileBytes;
        const unsigned char* al = ah + kTcTileBytes;
        const uint32_t dcol = tmem + 32u * gg;
#pragma unroll
        for (int pass = 0; pass < 3; ++pass) {
          const unsigned char* A = pass == 2 ? al : ah;
          const unsigned char* B = pass == 1 ? bl : bh;
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            const uint64_t da = tc_desc(smem_u32(A + 256 * ks), 128, 512);
            const uint64_t db = tc_desc(smem_u32(B + 256 * ks), 128, 512);
            const uint32_t acc = (pass | ks) ? 1u : 0u;
            asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                         "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                         ::"r"(dcol), "l"(da), "l"(db), "r"(idesc), "r"(acc) : "memory");
          }
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                   : "memory");
    }
    if (!wait_phase()) {
      timed_out = true;
      if (flags) atomicOr(flags, kFlagTcTimeout);
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    uint32_t r[32];
    const uint32_t taddr = tmem + ((uint32_t)((t >> 5) & 3) * 32u << 16) + 32u * g;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                 "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
                 "[%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                   "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                   "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = make_float2(__uint_as_float(r[2 * k]), __uint_as_float(r[2 * k + 1]));
  }

  // End of the kernel, every thread: after a timed-out wait, waits once more (bounded) for the outstanding MMAs,
  // then warp 0 frees the TMEM columns.
  __device__ __forceinline__ void teardown() {
    if (timed_out) {
      phase ^= 1u;
      wait_phase();
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
  }
};

// Host: the four B tiles (forward hi, forward lo, inverse hi, inverse lo) in the shared-memory tile layout, as
// bf16 bit patterns: B[2n + a][2k + b] of the angle D 2 pi n k / 16, split in double as hi = bf16(b), lo = bf16(b - hi)
// (round to nearest even).
inline uint16_t host_bf16_rn(double x) {
  float f = (float)x;
  uint32_t u;
  __builtin_memcpy(&u, &f, 4);
  const uint32_t rounding = 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)((u + rounding) >> 16);
}
inline double host_bf16_value(uint16_t h) {
  const uint32_t u = (uint32_t)h << 16;
  float f;
  __builtin_memcpy(&f, &u, 4);
  return (double)f;
}
inline void host_tc_btables(uint16_t* out /* kTcBBytes / 2 values */) {
  const double pi = 3.14159265358979323846;
  for (int dir = 0; dir < 2; ++dir) {
    const double D = dir == 0 ? -1.0 : 1.0;
    uint16_t* hi = out + (size_t)dir * 2 * (kTcBTileBytes / 2);
    uint16_t* lo = hi + kTcBTileBytes / 2;
    for (int n = 0; n < 16; ++n)
      for (int k = 0; k < 16; ++k) {
        const int m = (n * k) % 16;
        const double th = D * 2.0 * pi * m / 16.0;
        const double c = (m % 4 == 0) ? (m == 0 ? 1.0 : (m == 8 ? -1.0 : 0.0)) : std::cos(th);
        const double s = (m % 4 == 0) ? (m == 4 ? D : (m == 12 ? -D : 0.0)) : std::sin(th);
        const double val[2][2] = {{c, s}, {-s, c}};    // [a: Re/Im of x_n][b: Re/Im of X_k]
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b) {
            const int kk = 2 * n + a, nn = 2 * k + b;       // K index, N index (the tile row)
            const uint16_t h = host_bf16_rn(val[a][b]);
            const uint16_t l = host_bf16_rn(val[a][b] - host_bf16_value(h));
            hi[tc_tile_offset(nn, kk) / 2] = h;
            lo[tc_tile_offset(nn, kk) / 2] = l;
          }
      }
  }
}

}  // namespace nlv
