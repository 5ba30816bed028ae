// noalloc.cu -- true relative residual ||b - A x|| / ||b|| without any device
// allocation.
//
// Who needs this: code that must not call cudaMalloc once it is running --
// for example a host application whose memory manager owns the whole device
// after start-up, or a solver loop with a fixed, audited memory footprint.
// The other
// entry points of this library allocate their work space at setup; this one
// keeps its work space (the residual vector and the partial sums of the two
// norms) in a fixed array that lives in the library's device image instead.
//
// The array is MGD_NOALLOC_MAX_N + 2 * kParts doubles (about 4 MiB).  Every
// GPU that loads the library holds it until the process exits.  Calls share
// it: two calls whose work overlaps on the GPU (different streams, or
// different host threads) race on it and give wrong results; serialise them.
// The contents left by the previous call are never read: every element used
// by a call is written by that call first.
//
// CUDA loads a library's device code lazily by default, so the first call on
// a device may make the driver load this file's module, and with it reserve
// the array; from then on no call allocates or frees device memory.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/mgdamg.h"

namespace {

constexpr int kParts = 608;      // partial sums per norm (4 blocks per SM on 152 SMs)
constexpr int kThreadsNA = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[MGD_NOALLOC_MAX_N + 2 * kParts];

std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {nullptr};

// r_i = b_i - sum_j a_ij x_j, stored in the scratch array
__global__ void k_na_residual(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                              const double* __restrict__ v, const double* __restrict__ b,
                              const double* __restrict__ x, double* __restrict__ r) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int p = rp[i]; p < rp[i + 1]; ++p) s += v[p] * x[ci[p]];
    r[i] = b[i] - s;
  }
}

// part[blk] = sum of r_i^2 over this block's elements, part[kParts + blk] = sum of b_i^2
__global__ void k_na_partials(int n, const double* __restrict__ r, const double* __restrict__ b,
                              double* __restrict__ part) {
  double sr = 0.0, sb = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    sr += r[i] * r[i];
    sb += b[i] * b[i];
  }
  __shared__ double shr[kThreadsNA / 32], shb[kThreadsNA / 32];
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    sb += __shfl_xor_sync(0xffffffffu, sb, o);
  }
  if ((threadIdx.x & 31) == 0) {
    shr[threadIdx.x >> 5] = sr;
    shb[threadIdx.x >> 5] = sb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int k = 0; k < kThreadsNA / 32; ++k) {
      a += shr[k];
      c += shb[k];
    }
    part[blockIdx.x] = a;
    part[kParts + blockIdx.x] = c;
  }
}

// out[0] = ||r||, out[1] = ||b||, out[2] = ||r|| / ||b|| (0 when b = 0)
__global__ void k_na_final(const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double shr[kThreadsNA], shb[kThreadsNA];
  double a = 0.0, c = 0.0;
  for (int k = threadIdx.x; k < kParts; k += blockDim.x) {
    a += part[k];
    c += part[kParts + k];
  }
  shr[threadIdx.x] = a;
  shb[threadIdx.x] = c;
  __syncthreads();
  for (int o = kThreadsNA / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      shr[threadIdx.x] += shr[threadIdx.x + o];
      shb[threadIdx.x] += shb[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double nr = sqrt(shr[0]), nb = sqrt(shb[0]);
    out[0] = nr;
    out[1] = nb;
    out[2] = nb > 0.0 ? nr / nb : 0.0;
  }
}

// Device address of the scratch array for the current device, looked up once
// per device (host code must not use the symbol itself as an address).
int scratch_for_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return MGD_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return MGD_ECUDA;
    }
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return MGD_OK;
}

}  // namespace

extern "C" int mgd_relres_noalloc(int n, const int* d_rowptr, const int* d_colidx, const double* d_vals,
                                  const double* d_b, const double* d_x, double* d_out, void* stream) {
  if (n < 1 || n > MGD_NOALLOC_MAX_N || !d_rowptr || !d_colidx || !d_vals || !d_b || !d_x || !d_out)
    return MGD_EINVAL;
  double* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != MGD_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* r = scratch;
  double* part = scratch + MGD_NOALLOC_MAX_N;
  int nb = (n + kThreadsNA - 1) / kThreadsNA;
  if (nb > 4096) nb = 4096;
  // an error left pending by earlier, unrelated work would otherwise be
  // reported as a failure of this call's launches
  (void)cudaGetLastError();
  k_na_residual<<<nb, kThreadsNA, 0, s>>>(n, d_rowptr, d_colidx, d_vals, d_b, d_x, r);
  k_na_partials<<<kParts, kThreadsNA, 0, s>>>(n, r, d_b, part);
  k_na_final<<<1, kThreadsNA, 0, s>>>(part, d_out);
  if (cudaGetLastError() != cudaSuccess) return MGD_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return MGD_ECUDA;
  }
  return MGD_OK;
}
