// Gridding of radial samples onto the Cartesian grid: the interpolation that Sec. 3.1 performs on the CPU before
// the reconstruction, here as nearest-neighbour gridding with averaging on the GPU.  Sample i of spoke s lies at
// t_i d_s, t_i = -n/2 + i/2 (i < 2n), d_s the spoke's unit direction (cos, sin); each coordinate goes to the grid
// point floor(v + 1/2), the sample is kept when both lie in [-n/2, n/2), and a grid point (row = ky, column = kx,
// natural order) holds the mean of its samples.  The assignment depends on the trajectory only, so it is built once
// on the host as a table of the samples of every grid point (in sample order); the kernel gathers and averages,
// without atomics, so the result does not depend on scheduling.
#include <cmath>
#include <cstdlib>
#include <new>
#include <string>
#include <vector>

#include "nlinv.h"
#include "kernels.cuh"

void nlv_set_global_error(const std::string& msg);

struct nlinv_gridder {
  int n = 0, nspokes = 0;
  int* off = nullptr;            // device, n*n + 1: the samples of grid point g are idx[off[g] .. off[g+1])
  int* idx = nullptr;            // device: sample indices s * 2n + i, grouped by grid point
  cudaStream_t stream = nullptr;
  bool own_stream = false;
};

namespace {

// y[j][g] = mean of the samples of grid point g for coil j (0 if none); mask[g] = 1 if it has any.
__global__ void grid_gather_kernel(const float2* __restrict__ samples, const int* __restrict__ off,
                                   const int* __restrict__ idx, int cells, int ncoils, int per_coil, float2* y,
                                   uint8_t* mask) {
  nlv::pdl_enter();
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= (long)ncoils * cells) return;
  const int j = (int)(t / cells), g = (int)(t % cells);
  const int lo = off[g], hi = off[g + 1];
  const float2* sj = samples + (size_t)j * per_coil;
  float2 acc = make_float2(0.f, 0.f);
  for (int k = lo; k < hi; ++k) acc = nlv::cadd(acc, sj[idx[k]]);
  const int cnt = hi - lo;
  y[t] = cnt > 0 ? make_float2(acc.x / (float)cnt, acc.y / (float)cnt) : make_float2(0.f, 0.f);
  if (j == 0) mask[g] = cnt > 0 ? 1 : 0;
}

nlinv_status gfail(nlinv_status s, const std::string& msg) {
  nlv_set_global_error(msg);
  return s;
}

void gridder_free(nlinv_gridder* g) {
  if (!g) return;
  if (g->stream) cudaStreamSynchronize(g->stream);
  if (g->off) cudaFree(g->off);
  if (g->idx) cudaFree(g->idx);
  if (g->own_stream && g->stream) cudaStreamDestroy(g->stream);
  delete g;
}

bool device_ptr(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

nlinv_status nlinv_gridder_create(int n, int nspokes, const double* directions, void* stream, nlinv_gridder** out) {
  if (!out) return gfail(NLINV_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 8 || n > 2048 || (n & 1)) return gfail(NLINV_EINVAL, "n must be even and in 8..2048");
  if (nspokes < 1 || nspokes > 4096 || !directions)
    return gfail(NLINV_EINVAL, "1 <= nspokes <= 4096 and a directions array are required");
  for (int s = 0; s < 2 * nspokes; ++s)
    if (!std::isfinite(directions[s])) return gfail(NLINV_EINVAL, "directions must be finite");
  // grid point of every sample (or -1), then a counting sort by grid point that keeps the sample order
  const int T = 2 * n, cells = n * n;
  std::vector<int> cell((size_t)nspokes * T, -1);
  std::vector<int> count(cells + 1, 0);
  for (int s = 0; s < nspokes; ++s) {
    const double c = directions[2 * s], sn = directions[2 * s + 1];
    for (int i = 0; i < T; ++i) {
      const double t = -0.5 * n + 0.5 * i;
      const long kx = (long)std::floor(t * c + 0.5), ky = (long)std::floor(t * sn + 0.5);
      if (kx < -n / 2 || kx >= n / 2 || ky < -n / 2 || ky >= n / 2) continue;
      const int g = (int)(((ky % n + n) % n) * n + (kx % n + n) % n);
      cell[(size_t)s * T + i] = g;
      ++count[g + 1];
    }
  }
  for (int g = 0; g < cells; ++g) count[g + 1] += count[g];
  std::vector<int> idx(count[cells] > 0 ? count[cells] : 1);
  std::vector<int> fill(count.begin(), count.end() - 1);
  for (size_t k = 0; k < cell.size(); ++k)
    if (cell[k] >= 0) idx[fill[cell[k]]++] = (int)k;
  nlinv_gridder* g = new (std::nothrow) nlinv_gridder();
  if (!g) return gfail(NLINV_ENOMEM, "host allocation failed");
  g->n = n;
  g->nspokes = nspokes;
  cudaError_t e = cudaSuccess;
  if (stream) {
    g->stream = (cudaStream_t)stream;
  } else {
    e = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking);
    g->own_stream = e == cudaSuccess;
    if (e != cudaSuccess) g->stream = nullptr;
  }
  if (e == cudaSuccess) e = cudaMalloc(&g->off, (size_t)(cells + 1) * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&g->idx, idx.size() * sizeof(int));
  if (e == cudaSuccess)
    e = cudaMemcpy(g->off, count.data(), (size_t)(cells + 1) * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(g->idx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaGetLastError();
    gridder_free(g);
    return gfail(e == cudaErrorMemoryAllocation ? NLINV_ENOMEM : NLINV_ECUDA,
                 std::string("nlinv_gridder_create: ") + cudaGetErrorString(e));
  }
  *out = g;
  return NLINV_OK;
}

nlinv_status nlinv_grid(nlinv_gridder* g, int ncoils, const nlinv_c32* samples, nlinv_c32* y_out,
                        uint8_t* mask_out) {
  if (!g) return gfail(NLINV_EINVAL, "gridder is NULL");
  if (ncoils < 1 || ncoils > 64) return gfail(NLINV_EINVAL, "ncoils must be in 1..64");
  if (!samples || !y_out || !mask_out) return gfail(NLINV_EINVAL, "samples, y_out and mask_out are required");
  if (!device_ptr(samples) || !device_ptr(y_out) || !device_ptr(mask_out))
    return gfail(NLINV_EINVAL, "samples, y_out and mask_out must be device pointers");
  const int cells = g->n * g->n;
  const long threads = (long)ncoils * cells;
  const int block = 256;
  const unsigned grid = (unsigned)((threads + block - 1) / block);
  grid_gather_kernel<<<grid, block, 0, g->stream>>>((const float2*)samples, g->off, g->idx, cells, ncoils,
                                                    g->nspokes * 2 * g->n, (float2*)y_out, mask_out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return gfail(NLINV_ECUDA, std::string("nlinv_grid: ") + cudaGetErrorString(e));
  return NLINV_OK;
}

nlinv_status nlinv_gridder_destroy(nlinv_gridder* g) {
  gridder_free(g);
  return NLINV_OK;
}

}  // extern "C"
