// lbm_reduce_static: the FP64 reductions of lbm_reduce for caller-owned
// population buffers, without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need these
// diagnostics: an application that hands out all GPU memory from its own pool
// and forbids runtime allocations after start-up, or a plug-in that only
// receives device pointers from its host and has no lbm_ctx of its own.  This
// entry point therefore keeps its scratch (one FP64 partial sum per block and
// quantity) in a file-scope device array of fixed size instead of calling
// cudaMalloc.  The caller still passes the inputs (f, g) and the output (4
// doubles in device memory).
#include <cuda_runtime.h>

#include "lbm.h"
#include "lbm_phases.cuh"

namespace {

constexpr int kCellsPerBlock = 8192;  // fixed partition: the result does not depend on the GPU
constexpr int kMaxBlocks = 4096;      // scratch of 4096 x 4 doubles = 128 KiB
constexpr int kThreadsNa = 256;

// Shared by every call on a device and kept by every GPU that loads the
// library until the process exits; each call overwrites the partials it uses.
static __device__ __align__(256) double g_reduce_scratch[kMaxBlocks * 4];

// cv, rho_v and inv_drho arrive rounded to FP32, as the context kernels hold them
__global__ void k_reduce_partials_static(const float* __restrict__ f, const float* __restrict__ g, long long N,
                                         float cv, float rho_v, float inv_drho, double* partial) {
  double a[4] = {0, 0, 0, 0};
  const long long c0 = (long long)blockIdx.x * kCellsPerBlock;
  const long long c1 = c0 + kCellsPerBlock < N ? c0 + kCellsPerBlock : N;
  for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
    float fl[19], gl[7];
#pragma unroll
    for (int i = 0; i < 19; ++i) fl[i] = __ldg(f + i * N + c);
#pragma unroll
    for (int i = 0; i < 7; ++i) gl[i] = __ldg(g + i * N + c);
    float rho, jx, jy, jz;
    lbm::sum19(fl, rho, jx, jy, jz);
    const float T = lbm::sum7(gl);
    bool fin = isfinite(rho) && isfinite(T);
#pragma unroll
    for (int i = 0; i < 19; ++i) fin = fin && isfinite(fl[i]);
#pragma unroll
    for (int i = 0; i < 7; ++i) fin = fin && isfinite(gl[i]);
    if (fin) {
      a[0] += (double)rho;
      a[1] += (double)rho * (double)cv * (double)T;
      const double phi = ((double)rho - (double)rho_v) * (double)inv_drho;
      a[2] += phi < 0 ? 0.0 : (phi > 1 ? 1.0 : phi);
    } else {
      a[3] += 1.0;
    }
  }
  __shared__ double sh[4][kThreadsNa / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double v = a[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[k][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double v = 0;
    for (int w = 0; w < kThreadsNa / 32; ++w) v += sh[threadIdx.x][w];
    partial[blockIdx.x * 4 + threadIdx.x] = v;  // every partial in use is written: nothing to clear
  }
}

__global__ void k_reduce_finish_static(const double* partial, int nblocks, double* out) {
  if (threadIdx.x < 4) {
    double v = 0;
    for (int b = 0; b < nblocks; ++b) v += partial[b * 4 + threadIdx.x];
    out[threadIdx.x] = v;
  }
}

// Device address of the scratch array on the current device, looked up on every
// call (the array's name is only a host-side stand-in in host code; the lookup is
// cheap, enqueues nothing and stays valid across a reset of the device).
int scratch_for_current_device(double** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_reduce_scratch) != cudaSuccess || !p) return LBM_ERR_CUDA;
  *out = static_cast<double*>(p);
  return LBM_OK;
}

}  // namespace

extern "C" int lbm_reduce_static(const float* f, const float* g, long long n_cells, double cv, double rho_v,
                                 double rho_l, double* out, void* stream) {
  if (!f || !g || !out || n_cells <= 0 || !(cv > 0) || !(rho_l > rho_v)) return LBM_ERR_ARG;
  const long long nblocks = (n_cells + kCellsPerBlock - 1) / kCellsPerBlock;
  if (nblocks > kMaxBlocks) return LBM_ERR_ARG;  // more than kMaxBlocks * kCellsPerBlock cells
  double* scratch = nullptr;
  int st = scratch_for_current_device(&scratch);
  if (st != LBM_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_reduce_partials_static<<<(int)nblocks, kThreadsNa, 0, s>>>(f, g, n_cells, (float)cv, (float)rho_v,
                                                               (float)(1.0 / (rho_l - rho_v)), scratch);
  k_reduce_finish_static<<<1, 32, 0, s>>>(scratch, (int)nblocks, out);
  return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}
