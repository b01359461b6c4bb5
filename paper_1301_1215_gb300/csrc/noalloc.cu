// nlinv_forward_noalloc: the forward operator F of include/nlinv.h without any device allocation.
//
// Who needs it: callers that may not allocate device memory at the time they apply F -- for instance a scanner's
// real-time loop that reserves all of its GPU memory up front and must not risk a cudaMalloc failing or stalling
// mid-series, or a host framework that owns every device allocation and hands this library only its buffers.
// Such callers cannot create an nlinv_ctx (nlinv_create allocates the workspace), so this entry point keeps its
// scratch -- the twiddle and Sobolev tables, the Omega-column transform buffer and the coil maps -- in one
// file-scope __device__ array of fixed size (kScratchBytes).  Every GPU that loads the library holds that array
// until the process exits.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "nlinv.h"
#include "sizes.cuh"

void nlv_set_global_error(const std::string& msg);

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;   // 16 MiB: covers 384 x 384 with 10 coils at fov = n/4
constexpr int kMaxDevices = 64;
constexpr int kMaxSide = 512;                          // largest grid side with a compiled transform

// Layout of the array: the tables first, at offsets fixed for every call (so that tables written by an earlier
// call with the same n and Sobolev parameters are found where this call looks for them, whatever its coil count
// and field of view), then the transform buffer T and the coil maps, whose sizes vary from call to call.
constexpr size_t kTwOff = 0;                                             // twiddles of the split (N1, N2)
constexpr size_t kTwBOff = kTwOff + size_t(kMaxSide) * 8;                // twiddles of the split (N2, N1)
constexpr size_t kWOff = kTwBOff + size_t(kMaxSide) * 8;                 // Sobolev weight, n x n floats
constexpr size_t kDataOff = kWOff + size_t(kMaxSide) * kMaxSide * 4;     // T, then the coil maps
static_assert(kDataOff % 256 == 0, "the data region must stay 256-byte aligned");

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Per-device host-side state: the device address of g_scratch and the key of the tables last written there.
struct DeviceState {
  bool ready = false;
  unsigned char* base = nullptr;
  int n = 0;
  double a = -1.0, l = -1.0;
};
std::mutex g_mutex;
DeviceState g_state[kMaxDevices];

size_t round256(size_t v) { return (v + 255) / 256 * 256; }

nlinv_status fail(nlinv_status s, const std::string& msg) {
  nlv_set_global_error(msg);
  return s;
}

// Device memory of device `dev` (the current device, which runs the kernels and holds the scratch array), or
// managed memory.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

cudaError_t launch(const void* fn, int grid, int block, size_t smem, cudaStream_t st, nlv::KArgs a) {
  void* args[] = {&a};
  return cudaLaunchKernel(fn, dim3(grid), dim3(block), args, smem, st);
}

}  // namespace

extern "C" NLINV_API nlinv_status nlinv_forward_noalloc(const nlinv_params* p, void* stream, const nlinv_c32* x,
                                                        const uint8_t* mask, nlinv_c32* y_out) {
  if (!p) return fail(NLINV_EINVAL, "params is NULL");
  const nlv::SizeKernels* k = nlv::find_size(p->n);
  if (!k) return fail(NLINV_EINVAL, "grid side n=" + std::to_string(p->n) + " has no compiled transform");
  if (p->ncoils < 1 || p->ncoils > 64) return fail(NLINV_EINVAL, "ncoils must be in 1..64");
  if (p->fov < 1 || p->fov > p->n / 2) return fail(NLINV_EINVAL, "fov must be in 1..n/2");
  if (!(p->sobolev_a >= 0) || !(p->sobolev_l >= 0) || !std::isfinite(p->sobolev_a) || !std::isfinite(p->sobolev_l))
    return fail(NLINV_EINVAL, "sobolev_a and sobolev_l must be finite and >= 0");
  if (!x || !mask || !y_out) return fail(NLINV_EINVAL, "x, mask and y_out must not be NULL");
  if (p->n > kMaxSide) return fail(NLINV_EINVAL, "grid side beyond the table region of the scratch array");

  const int N = p->n, J = p->ncoils, f = p->fov, Wc = 2 * f;
  const size_t plane = (size_t)N * N;
  const size_t bT = round256((size_t)J * N * Wc * sizeof(float2));
  const size_t bC = round256((size_t)J * Wc * Wc * sizeof(float2));
  const size_t need = kDataOff + bT + bC;
  if (need > kScratchBytes)
    return fail(NLINV_EINVAL, "nlinv_forward_noalloc needs " + std::to_string(need) +
                                  " bytes of scratch for this n, ncoils and fov; its static maximum is " +
                                  std::to_string(kScratchBytes) + " bytes (use nlinv_create + nlinv_forward)");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(NLINV_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(NLINV_EINVAL, "device ordinal out of range");
  if (!on_device(x, dev) || !on_device(mask, dev) || !on_device(y_out, dev))
    return fail(NLINV_EINVAL, "x, mask and y_out must be device (or managed) memory of the current device");
  cudaStream_t st = (cudaStream_t)stream;

  std::lock_guard<std::mutex> lock(g_mutex);
  DeviceState& ds = g_state[dev];
  if (!ds.ready) {
    // once per device, with that device current: the device address of the file-scope scratch array
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_scratch);
    if (e != cudaSuccess) return fail(NLINV_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    ds.base = (unsigned char*)ptr;
    ds.ready = true;
  }
  unsigned char* b = ds.base;
  float2* twA = (float2*)(b + kTwOff);
  float2* twB = (float2*)(b + kTwBOff);
  float* wtab = (float*)(b + kWOff);
  float2* T = (float2*)(b + kDataOff);
  float2* coil = (float2*)(b + kDataOff + bT);

  if (ds.n != N || ds.a != p->sobolev_a || ds.l != p->sobolev_l) {
    // tables for this grid side and weight: computed here, copied into the scratch array, then the stream is
    // waited for so that the host buffers may go away
    const int N1 = k->N1, N2 = k->N2;
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
    std::vector<float> wt(plane);
    for (int k1 = 0; k1 < N; ++k1)
      for (int k2 = 0; k2 < N; ++k2) {
        const double g1 = k1 < N / 2 ? k1 : k1 - N, g2 = k2 < N / 2 ? k2 : k2 - N;
        wt[(size_t)k1 * N + k2] =
            (float)std::pow(1.0 + p->sobolev_a * (g1 * g1 + g2 * g2) / ((double)N * N), -0.5 * p->sobolev_l);
      }
    e = cudaMemcpyAsync(twA, ta.data(), N * sizeof(float2), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(twB, tb.data(), N * sizeof(float2), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(wtab, wt.data(), plane * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      ds.n = 0;
      return fail(NLINV_ECUDA, std::string("table upload: ") + cudaGetErrorString(e));
    }
    ds.n = N;
    ds.a = p->sobolev_a;
    ds.l = p->sobolev_l;
  }

  int smem_optin = 0;
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  for (const void* fn : {k->row[nlv::ROW_W_IFFT], k->row[nlv::ROW_FFT_P_OUT], k->col[nlv::COL_IFFT_C],
                         k->col[nlv::COL_PROD_FFT]}) {
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, fn) == cudaSuccess)
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin - (int)fa.sharedSizeBytes);
  }
  cudaGetLastError();

  // the same four passes as nlinv_forward, on the scratch array instead of a context workspace
  nlv::KArgs a{};
  a.N = N; a.J = J; a.f = f; a.Wc = Wc;
  a.wtab = wtab; a.twA = twA; a.twB = twB;
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const nlv::RowGrid rg = nlv::row_grid(k, J * N, 0, sms < 1 ? 1 : sms, nlv::kRowCtasPerSM);
  const int cols = J * ((Wc + k->col_lanes - 1) / k->col_lanes);
  const float2* xv = (const float2*)x;

  nlv::KArgs a1 = a;                        // T = FFT^-1_row(w chat_j), Omega columns
  a1.src = xv + plane; a1.dst = T; a1.nrows = J * N; a1.rows_per_cta = rg.rows_per_cta;
  e = launch(k->row[nlv::ROW_W_IFFT], rg.blocks, rg.lanes * k->tl, k->row_smem(nlv::ROW_W_IFFT, rg.lanes), st, a1);
  nlv::KArgs a2 = a;                        // c_j = Omega rows of FFT^-1_col(T)
  a2.src = T; a2.dst = coil; a2.nrows = J;
  if (e == cudaSuccess) e = launch(k->col[nlv::COL_IFFT_C], cols, k->col_threads, k->col_smem(nlv::COL_IFFT_C, Wc), st, a2);
  nlv::KArgs a3 = a;                        // T = FFT_col(M rho c_j)
  a3.rho = xv; a3.coil = coil; a3.dst = T; a3.nrows = J;
  if (e == cudaSuccess) e = launch(k->col[nlv::COL_PROD_FFT], cols, k->col_threads, k->col_smem(nlv::COL_PROD_FFT, Wc), st, a3);
  nlv::KArgs a4 = a;                        // y = P FFT_row(T)
  a4.src = T; a4.dst = (float2*)y_out; a4.mask = mask; a4.nrows = J * N; a4.rows_per_cta = rg.rows_per_cta;
  if (e == cudaSuccess)
    e = launch(k->row[nlv::ROW_FFT_P_OUT], rg.blocks, rg.lanes * k->tl, k->row_smem(nlv::ROW_FFT_P_OUT, rg.lanes), st,
               a4);
  if (e != cudaSuccess) return fail(NLINV_ECUDA, std::string("nlinv_forward_noalloc: ") + cudaGetErrorString(e));
  return NLINV_OK;
}
