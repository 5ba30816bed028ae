// solve_kernels.cu -- device kernels of the solve phase outside the V-cycle:
// the block-level updates of the block preconditioners (Sections 3.3-3.4),
// generic SpMV / residual, and the FGMRES vector work.  All are HBM-bound
// streaming or sparse kernels.
#include "../../include/mgdamg.h"
#include "mgd_internal.cuh"
#include "row_dot.cuh"

#include <cooperative_groups.h>

#include <functional>

namespace mgd {

namespace cg = cooperative_groups;

// ---------------------------------------------------------------- binary32 <-> binary64
// The block updates of the FP32-V-cycle form convert every V-cycle input and
// output between the IEEE-754 binary32 and binary64 formats.  On this part
// the conversion instruction issues on the FP64 pipe, which already bounds
// these updates, so the common cases are done on the integer pipe from the
// formats' definitions (IEEE 754-2008, 3.4 and 5.4.2; round to nearest, ties
// to even): a normal binary32 widens exactly by rebiasing its exponent (127 ->
// 1023) and shifting its 23-bit significand up by 29; a binary64 whose value
// lies in the binary32 normal range keeps its top 23 significand bits and is
// rounded on the remaining 29 (a carry out of the significand moves to the
// next binade, and out of the largest one to infinity).  Zeros are built
// directly; subnormal, infinite and NaN operands, and binary64 values outside
// the binary32 normal range, take the hardware conversion.
// mgd_check_conversions compares both with the hardware conversion.

// the hardware conversions of the rare operands, out of line so that the
// common path does not issue them predicated off
__device__ __noinline__ double f32_to_f64_hw(float f) { return (double)f; }
__device__ __noinline__ float f64_to_f32_hw(double d) { return (float)d; }

__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  if ((u & 0x7fffffffu) == 0) return __longlong_as_double((long long)sign);
  if (e == 0 || e == 255) return f32_to_f64_hw(f);
  return __longlong_as_double(
      (long long)(sign | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29)));
}

__device__ __forceinline__ float f64_to_f32(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned sign = (unsigned)(b >> 63) << 31;
  if ((b << 1) == 0) return __uint_as_float(sign);
  const int fe = (int)((b >> 52) & 0x7ffu) - 896;  // binary32 exponent field if normal
  if (fe < 1 || fe > 254) return f64_to_f32_hw(d);
  const unsigned keep = (unsigned)((b >> 29) & 0x7fffffu);
  const unsigned rem = (unsigned)(b & 0x1fffffffu);
  unsigned r = ((unsigned)fe << 23) | keep;
  if (rem > 0x10000000u || (rem == 0x10000000u && (keep & 1u))) ++r;
  return __uint_as_float(sign | r);
}

__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return f32_to_f64(x); }
template <typename T>
__device__ __forceinline__ T from_f64(double x);
template <>
__device__ __forceinline__ double from_f64<double>(double x) {
  return x;
}
template <>
__device__ __forceinline__ float from_f64<float>(double x) {
  return f64_to_f32(x);
}

// s x for a consume coefficient: +1 and -1 (every coefficient of the block
// preconditioners, flagged on the host) without a multiply; the same bits
__device__ __forceinline__ double unit_times(int unit, double s, double x) {
  if (unit == 1) return x;
  if (unit == 2) return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
  return s * x;
}

// ---------------------------------------------------------------- block-level updates
__device__ __forceinline__ double* resolve(const PRef& r, const IOSlots* io) {
  if (r.slot == 0) return r.abs;
  if (r.slot == 1) return const_cast<double*>(io->v) + r.off;
  return io->z + r.off;
}

// dst = (T)(a + sum_t s_t d_t (.) w_t)
template <typename T>
__global__ void k_produce(const ProduceDesc<T>* __restrict__ ds, int N, const IOSlots* __restrict__ io) {
  MGD_PDL_ENTRY();
  const ProduceDesc<T>* d = ds + blockIdx.y;
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const double* a = resolve(d->a, io);
  double acc = a ? a[k] : 0.0;
  int nt = d->nt;
  for (int t = 0; t < nt; ++t) {
    const double* w = resolve(d->w[t], io);
    double term = w[k];
    if (d->d[t]) term *= d->d[t][k];
    acc += d->s[t] * term;
  }
  d->dst[k] = from_f64<T>(acc);
}

// dst = base + s * x
template <typename T>
__global__ void k_consume(const ConsumeDesc<T>* __restrict__ ds, int N, const IOSlots* __restrict__ io) {
  MGD_PDL_ENTRY();
  const ConsumeDesc<T>* d = ds + blockIdx.y;
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  double* dst = resolve(d->dst, io);
  const double* base = resolve(d->base, io);
  double val = unit_times(d->unit, d->s, to_f64(d->x[k]));
  dst[k] = base ? base[k] + val : val;
}

// A CONSUME step followed by a PRODUCE step, fused: per element, every
// consume descriptor, then every produce descriptor, each computed as in
// k_consume / k_produce.  The block first resolves the descriptors' vectors
// into shared memory.  The descriptors of one step are independent (those
// kernels run them as parallel blocks), so a thread issues the loads of
// kCpGroup descriptors (or of kCpGroup terms of one descriptor) before it uses
// them or stores a result: one descriptor at a time would leave a single
// dependent load per thread in flight.  A produce term that reads a vector
// the consume just wrote reads it back at the same index in the same thread,
// after the store (the data pointers are not restrict: the compiler keeps the
// order).  The host fuses only steps within the shared-memory tables' sizes.
constexpr int kCpGroup = 4;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_consume_produce(const ConsumeDesc<T>* __restrict__ cd, int ncd,
                                                              const ProduceDesc<T>* __restrict__ pd, int npd, int N,
                                                              const IOSlots* __restrict__ io) {
  __shared__ const T* s_cx[kCpMaxCons];
  __shared__ const double* s_cb[kCpMaxCons];
  __shared__ double* s_cdst[kCpMaxCons];
  __shared__ double s_cs[kCpMaxCons];
  __shared__ int s_cu[kCpMaxCons];
  __shared__ T* s_pdst[kCpMaxProd];
  __shared__ const double* s_pa[kCpMaxProd];
  __shared__ int s_pt[kCpMaxProd + 1];  // terms of produce j: [s_pt[j], s_pt[j+1])
  __shared__ const double* s_tw[kCpMaxTerms];
  __shared__ const double* s_td[kCpMaxTerms];
  __shared__ double s_ts[kCpMaxTerms];
  MGD_PDL_ENTRY();
  const int t = threadIdx.x;
  for (int j = t; j < ncd; j += blockDim.x) {
    const ConsumeDesc<T>* d = cd + j;
    s_cx[j] = d->x;
    s_cb[j] = resolve(d->base, io);
    s_cdst[j] = resolve(d->dst, io);
    s_cs[j] = d->s;
    s_cu[j] = d->unit;
  }
  for (int j = t; j < npd; j += blockDim.x) {
    const ProduceDesc<T>* d = pd + j;
    int o = 0;
    for (int q = 0; q < j; ++q) o += pd[q].nt;
    s_pdst[j] = d->dst;
    s_pa[j] = resolve(d->a, io);
    s_pt[j] = o;
    for (int u = 0; u < d->nt; ++u) {
      s_tw[o + u] = resolve(d->w[u], io);
      s_td[o + u] = d->d[u];
      s_ts[o + u] = d->s[u];
    }
    if (j == npd - 1) s_pt[npd] = o + d->nt;
  }
  __syncthreads();
  const int k = blockIdx.x * blockDim.x + t;
  if (k >= N) return;
  for (int j0 = 0; j0 < ncd; j0 += kCpGroup) {
    double xv[kCpGroup], bv[kCpGroup];
#pragma unroll
    for (int u = 0; u < kCpGroup; ++u) {
      xv[u] = 0.0;
      bv[u] = 0.0;
      if (j0 + u < ncd) {
        xv[u] = to_f64(s_cx[j0 + u][k]);
        const double* b = s_cb[j0 + u];
        if (b) bv[u] = b[k];
      }
    }
#pragma unroll
    for (int u = 0; u < kCpGroup; ++u)
      if (j0 + u < ncd) {
        const int j = j0 + u;
        double val = unit_times(s_cu[j], s_cs[j], xv[u]);
        s_cdst[j][k] = s_cb[j] ? bv[u] + val : val;
      }
  }
  for (int j = 0; j < npd;) {
    if (s_pt[j + 1] - s_pt[j] <= 1) {
      // up to kCpGroup consecutive descriptors with at most one term each
      int m = 1;
      while (m < kCpGroup && j + m < npd && s_pt[j + m + 1] - s_pt[j + m] <= 1) ++m;
      double av[kCpGroup], wv[kCpGroup], dv[kCpGroup];
#pragma unroll
      for (int u = 0; u < kCpGroup; ++u) {
        av[u] = 0.0;
        wv[u] = 0.0;
        dv[u] = 1.0;
        if (u < m) {
          const double* a = s_pa[j + u];
          if (a) av[u] = a[k];
          const int o = s_pt[j + u];
          if (s_pt[j + u + 1] > o) {
            wv[u] = s_tw[o][k];
            const double* dd = s_td[o];
            if (dd) dv[u] = dd[k];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < kCpGroup; ++u)
        if (u < m) {
          double acc = av[u];
          const int o = s_pt[j + u];
          if (s_pt[j + u + 1] > o) {
            double term = wv[u];
            if (s_td[o]) term *= dv[u];
            acc += s_ts[o] * term;
          }
          s_pdst[j + u][k] = from_f64<T>(acc);
        }
      j += m;
    } else {
      const int o0 = s_pt[j], o1 = s_pt[j + 1];
      const double* a = s_pa[j];
      double acc = a ? a[k] : 0.0;
      for (int o = o0; o < o1; o += kCpGroup) {
        double wv[kCpGroup], dv[kCpGroup];
#pragma unroll
        for (int q = 0; q < kCpGroup; ++q) {
          wv[q] = 0.0;
          dv[q] = 1.0;
          if (o + q < o1) {
            wv[q] = s_tw[o + q][k];
            const double* dd = s_td[o + q];
            if (dd) dv[q] = dd[k];
          }
        }
#pragma unroll
        for (int q = 0; q < kCpGroup; ++q)
          if (o + q < o1) {
            double term = wv[q];
            if (s_td[o + q]) term *= dv[q];
            acc += s_ts[o + q] * term;
          }
      }
      s_pdst[j][k] = from_f64<T>(acc);
      ++j;
    }
  }
}

template <typename T>
void launch_consume_produce(const ConsumeDesc<T>* cd, int ncd, const ProduceDesc<T>* pd, int npd, int N,
                            const IOSlots* io, cudaStream_t s) {
  if (N <= 0) return;
  launch_k(k_consume_produce<T>, dim3(cdiv(N, kThreads)), dim3(kThreads), 0, s, cd, ncd, pd, npd, N, io);
  MGD_LAUNCH_CHECK();
}
template void launch_consume_produce<double>(const ConsumeDesc<double>*, int, const ProduceDesc<double>*, int, int,
                                             const IOSlots*, cudaStream_t);
template void launch_consume_produce<float>(const ConsumeDesc<float>*, int, const ProduceDesc<float>*, int, int,
                                            const IOSlots*, cudaStream_t);

// FP64 issue-rate reference: four independent multiply-add chains per thread
// and enough warps to fill every SM; the peak of the FP64 roofline (lane
// operations per second with every lane active)
__global__ void __launch_bounds__(512) k_fp64_rate(int iters, double* out) {
  double a = 1.0 + threadIdx.x * 1e-9, b = 0.999999, c0 = 1e-7, c1 = 2e-7, c2 = 3e-7, c3 = 4e-7;
  for (int i = 0; i < iters; ++i) {
    c0 = fma(a, b, c0);
    c1 = fma(a, b, c1);
    c2 = fma(a, b, c2);
    c3 = fma(a, b, c3);
  }
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = c0 + c1 + c2 + c3;
}

double measure_fp64_rate(cudaStream_t s) {
  int dev = 0, nsm = 0;
  MGD_CUDA(cudaGetDevice(&dev));
  MGD_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int threads = 512, blocks = 4 * nsm, iters = 4096;
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms = 0.f;
  cudaError_t e = cudaMallocAsync(&out, sizeof(double) * blocks * threads, s);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    k_fp64_rate<<<blocks, threads, 0, s>>>(iters, out);  // warm-up
    cudaEventRecord(e0, s);
    k_fp64_rate<<<blocks, threads, 0, s>>>(iters, out);
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  }
  if (out) cudaFreeAsync(out, s);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess || ms <= 0.f) throw Error{MGD_ECUDA, "FP64 rate measurement failed"};
  return (double)blocks * threads * iters * 4.0 / (ms * 1e-3);
}

// Self-check of f32_to_f64 / f64_to_f32 against the hardware conversions:
// every binary32 pattern widened; and narrowed, for every binary32 value f, f
// itself, the midpoint between f and the next binary32 above it (a tie) and
// the binary64 neighbours of that midpoint.  NaN results compare as equal
// when both are NaN.
__device__ __forceinline__ bool same_f64(double a, double b) {
  return __double_as_longlong(a) == __double_as_longlong(b) || (isnan(a) && isnan(b));
}
__device__ __forceinline__ bool same_f32(float a, float b) {
  return __float_as_uint(a) == __float_as_uint(b) || (isnan(a) && isnan(b));
}

__global__ void k_check_conversions(unsigned long long* mismatches) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  unsigned long long bad = 0;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < (1ull << 32); i += stride) {
    const unsigned u = (unsigned)i;
    const float f = __uint_as_float(u);
    const double w = (double)f;
    if (!same_f64(f32_to_f64(f), w)) ++bad;
    if (!same_f32(f64_to_f32(w), (float)w)) ++bad;
    if ((u & 0x7f800000u) != 0x7f800000u && (u & 0x7fffffffu) != 0x7f7fffffu) {
      // the next binary32 away from zero is finite: the midpoint is exact in binary64
      const double up = (double)__uint_as_float(u + 1u);
      const double mid = 0.5 * (w + up);
      const long long mb = __double_as_longlong(mid);
      const double lo = __longlong_as_double(mb - 1), hi = __longlong_as_double(mb + 1);
      if (!same_f32(f64_to_f32(mid), (float)mid)) ++bad;
      if (!same_f32(f64_to_f32(lo), (float)lo)) ++bad;
      if (!same_f32(f64_to_f32(hi), (float)hi)) ++bad;
    }
  }
  if (bad) atomicAdd(mismatches, bad);
}

long long check_conversions(cudaStream_t s) {
  int dev = 0, nsm = 0;
  MGD_CUDA(cudaGetDevice(&dev));
  MGD_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  unsigned long long* d = nullptr;
  unsigned long long h = 0;
  cudaError_t e = cudaMallocAsync(&d, sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) {
    k_check_conversions<<<8 * nsm, 256, 0, s>>>(d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (d) {
    cudaFreeAsync(d, s);
    cudaStreamSynchronize(s);
  }
  if (e != cudaSuccess) throw Error{MGD_ECUDA, "conversion check failed"};
  return (long long)h;
}

template <typename T>
__global__ void k_jacobi(const JacDesc<T>* __restrict__ ds, int N) {
  MGD_PDL_ENTRY();
  const JacDesc<T>* d = ds + blockIdx.y;
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < N) d->x[k] = d->dinv[k] * d->b[k];
}

template <typename T>
void launch_produce(const ProduceDesc<T>* d, int nd, int N, const IOSlots* io, cudaStream_t s) {
  if (nd <= 0) return;
  launch_k(k_produce<T>, dim3(dim3(cdiv(N, kThreads), nd)), dim3(kThreads), 0, s, d, N, io);
  MGD_LAUNCH_CHECK();
}
template <typename T>
void launch_consume(const ConsumeDesc<T>* d, int nd, int N, const IOSlots* io, cudaStream_t s) {
  if (nd <= 0) return;
  launch_k(k_consume<T>, dim3(dim3(cdiv(N, kThreads), nd)), dim3(kThreads), 0, s, d, N, io);
  MGD_LAUNCH_CHECK();
}
template <typename T>
void launch_jacobi(const JacDesc<T>* d, int nd, int N, cudaStream_t s) {
  if (nd <= 0) return;
  launch_k(k_jacobi<T>, dim3(dim3(cdiv(N, kThreads), nd)), dim3(kThreads), 0, s, d, N);
  MGD_LAUNCH_CHECK();
}
template void launch_produce<double>(const ProduceDesc<double>*, int, int, const IOSlots*, cudaStream_t);
template void launch_produce<float>(const ProduceDesc<float>*, int, int, const IOSlots*, cudaStream_t);
template void launch_consume<double>(const ConsumeDesc<double>*, int, int, const IOSlots*, cudaStream_t);
template void launch_consume<float>(const ConsumeDesc<float>*, int, int, const IOSlots*, cudaStream_t);
template void launch_jacobi<double>(const JacDesc<double>*, int, int, cudaStream_t);
template void launch_jacobi<float>(const JacDesc<float>*, int, int, cudaStream_t);

// ---------------------------------------------------------------- generic residual / SpMV
template <typename T, int FMT, int MODE>  // MODE 0: y = A x ; 1: r = b - A x
__global__ void __launch_bounds__(kThreads) k_spmv(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                                   const T* __restrict__ v, const int* __restrict__ sptr,
                                                   const int* __restrict__ sci, const T* __restrict__ sv,
                                                   const T* __restrict__ b, const T* __restrict__ x,
                                                   T* __restrict__ y) {
  MGD_PDL_TRIGGER();  // the operator is setup-time data: load its rows before the wait
  constexpr int TPR = FmtTraits<FMT>::tpr;
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int row = (int)(g / TPR), lane = (int)(g % TPR);
  if (((g & ~31LL) / TPR) >= n) return;
  bool valid = row < n;
  RowPre<T, 4> R;
  row_load<T, FMT, 4>(R, row, lane, valid, rp, ci, v, sptr, sci, sv);
  MGD_PDL_WAIT();
  XPlain<T> xf{x};
  T s = row_finish<T, FMT, 4>(R, valid, ci, v, sci, sv, xf);
  if (valid && lane == 0) y[row] = MODE ? b[row] - s : s;
}

template <typename T, int MODE>
static void spmv_dispatch(int fmt, int n, const int* rp, const int* ci, const T* v, const int* sptr,
                          const int* sci, const T* sv, const T* b, const T* x, T* y, cudaStream_t s) {
  if (n <= 0) return;
  if (fmt == FMT_SELL && !sptr) fmt = FMT_CSR4;
  auto g = [&](int tpr) { return cdiv((long long)n * tpr + 32, kThreads); };
  switch (fmt) {
    case FMT_SELL: launch_k(k_spmv<T, FMT_SELL, MODE>, dim3(g(1)), dim3(kThreads), 0, s, n, rp, ci, v, sptr, sci, sv, b, x, y); break;
    case FMT_CSR1: launch_k(k_spmv<T, FMT_CSR1, MODE>, dim3(g(1)), dim3(kThreads), 0, s, n, rp, ci, v, sptr, sci, sv, b, x, y); break;
    case FMT_CSR2: launch_k(k_spmv<T, FMT_CSR2, MODE>, dim3(g(2)), dim3(kThreads), 0, s, n, rp, ci, v, sptr, sci, sv, b, x, y); break;
    case FMT_CSR4: launch_k(k_spmv<T, FMT_CSR4, MODE>, dim3(g(4)), dim3(kThreads), 0, s, n, rp, ci, v, sptr, sci, sv, b, x, y); break;
    case FMT_CSR8: launch_k(k_spmv<T, FMT_CSR8, MODE>, dim3(g(8)), dim3(kThreads), 0, s, n, rp, ci, v, sptr, sci, sv, b, x, y); break;
    case FMT_CSR16:
      launch_k(k_spmv<T, FMT_CSR16, MODE>, dim3(g(16)), dim3(kThreads), 0, s, n, rp, ci, v, sptr, sci, sv, b, x, y);
      break;
    default: launch_k(k_spmv<T, FMT_CSR32, MODE>, dim3(g(32)), dim3(kThreads), 0, s, n, rp, ci, v, sptr, sci, sv, b, x, y); break;
  }
  MGD_LAUNCH_CHECK();
}

template <typename T>
void launch_residual(int fmt, int n, const int* rp, const int* ci, const T* v, const int* sptr, const int* sci,
                     const T* sv, const T* b, const T* x, T* r, cudaStream_t s) {
  spmv_dispatch<T, 1>(fmt, n, rp, ci, v, sptr, sci, sv, b, x, r, s);
}
template void launch_residual<double>(int, int, const int*, const int*, const double*, const int*, const int*,
                                      const double*, const double*, const double*, double*, cudaStream_t);
template void launch_residual<float>(int, int, const int*, const int*, const float*, const int*, const int*,
                                     const float*, const float*, const float*, float*, cudaStream_t);

void launch_spmv_f64(int fmt, int n, const int* rp, const int* ci, const double* v, const int* sptr,
                     const int* sci, const double* sv, const double* x, double* y, cudaStream_t s) {
  spmv_dispatch<double, 0>(fmt, n, rp, ci, v, sptr, sci, sv, nullptr, x, y, s);
}
void launch_resid_f64(int fmt, int n, const int* rp, const int* ci, const double* v, const int* sptr,
                      const int* sci, const double* sv, const double* b, const double* x, double* r,
                      cudaStream_t s) {
  spmv_dispatch<double, 1>(fmt, n, rp, ci, v, sptr, sci, sv, b, x, r, s);
}

template <typename T>
__global__ void k_axpy(int n, T* y, const T* x) {
  MGD_PDL_ENTRY();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += x[i];
}
template <typename T>
void launch_axpy(int n, T* y, const T* x, cudaStream_t s) {
  if (n <= 0) return;
  launch_k(k_axpy<T>, dim3(cdiv(n, kThreads)), dim3(kThreads), 0, s, n, y, x);
  MGD_LAUNCH_CHECK();
}
template void launch_axpy<double>(int, double*, const double*, cudaStream_t);
template void launch_axpy<float>(int, float*, const float*, cudaStream_t);

__global__ void k_set_io(IOSlots* io, const double* v, double* z) {
  MGD_PDL_ENTRY();
  io->v = v;
  io->z = z;
}
void launch_set_io(IOSlots* io, const double* v, double* z, cudaStream_t s) {
  launch_k(k_set_io, dim3(1), dim3(1), 0, s, io, v, z);
  MGD_LAUNCH_CHECK();
}

__global__ void k_cast_df(int n, const double* a, float* b) {
  MGD_PDL_ENTRY();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}
__global__ void k_cast_fd(int n, const float* a, double* b) {
  MGD_PDL_ENTRY();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}
__global__ void k_copy(int n, const double* a, double* b) {
  MGD_PDL_ENTRY();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = a[i];
}
void launch_cast_f64_f32(int n, const double* a, float* b, cudaStream_t s) {
  if (n <= 0) return;
  launch_k(k_cast_df, dim3(cdiv(n, kThreads)), dim3(kThreads), 0, s, n, a, b);
  MGD_LAUNCH_CHECK();
}
void launch_cast_f32_f64(int n, const float* a, double* b, cudaStream_t s) {
  if (n <= 0) return;
  launch_k(k_cast_fd, dim3(cdiv(n, kThreads)), dim3(kThreads), 0, s, n, a, b);
  MGD_LAUNCH_CHECK();
}
void launch_copy_f64(int n, const double* a, double* b, cudaStream_t s) {
  if (n <= 0) return;
  launch_k(k_copy, dim3(cdiv(n, kThreads)), dim3(kThreads), 0, s, n, a, b);
  MGD_LAUNCH_CHECK();
}

// ---------------------------------------------------------------- Arnoldi (FP64)
constexpr int kMaxV = 32;

// out[t] = sum_b partial[b * kMaxV + t]  (fixed order: deterministic)
__global__ void k_reduce_partials(const double* __restrict__ partial, int nblocks, int nv, double* __restrict__ out) {
  MGD_PDL_ENTRY();
  int t = blockIdx.x;
  if (t >= nv) return;
  __shared__ double sh[kThreads];
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partial[(size_t)b * kMaxV + t];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[t] = sh[0];
}

static int dot_blocks(int n) { return std::min(kDotBlocks, std::max(1, cdiv(n, kThreads))); }

// Modified Gram-Schmidt, one fused pass per basis vector (the orthogonalisation
// the oracle uses, Saad's MGS-Arnoldi): step i reads the partial sums of
// <v_i, w> left by the previous pass, forms h_i (every block reduces them in
// the same fixed order, so all blocks agree bit for bit), updates
// w -= h_i v_i and accumulates the partial sums of <v_{i+1}, w> -- or of
// <w, w> after the last vector.  Two FP64 multiply-adds per element per basis
// vector, which on this part's FP64 rate is what the orthogonalisation costs.
__global__ void __launch_bounds__(kThreads) k_dot_partial(int n, const double* __restrict__ a,
                                                          const double* __restrict__ b,
                                                          double* __restrict__ partial) {
  MGD_PDL_ENTRY();
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s += a[i] * b[i];
  __shared__ double sh[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) t += sh[k];
    partial[blockIdx.x] = t;
  }
}

__device__ __forceinline__ double block_sum_partials(const double* __restrict__ partial, int nb) {
  __shared__ double sh[kThreads];
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += partial[b];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kThreads) k_mgs_step(int n, const double* __restrict__ vi,
                                                       const double* __restrict__ vnext, double* __restrict__ w,
                                                       const double* __restrict__ pin, int nb,
                                                       double* __restrict__ pout, double* __restrict__ hout) {
  MGD_PDL_ENTRY();
  const double h = block_sum_partials(pin, nb);
  if (blockIdx.x == 0 && threadIdx.x == 0) *hout = h;
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double wi = w[i] - h * vi[i];
    w[i] = wi;
    s += (vnext ? vnext[i] : wi) * wi;
  }
  __shared__ double sh[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) t += sh[k];
    pout[blockIdx.x] = t;
  }
}

// The same two kernels on 16-byte vectors: every thread keeps kMgsU pairs of
// each stream in flight per trip (the scalar loop above has one element of
// each, too few bytes in flight per SM to cover HBM latency).  Used when n is
// even and every vector starts on a 16-byte boundary; the sums run in a fixed
// order per (n, grid), so every run gives the same bits.
constexpr int kMgsU = 2;

__global__ void __launch_bounds__(kThreads) k_dot_partial2(int n2, const double2* __restrict__ a,
                                                           const double2* __restrict__ b,
                                                           double* __restrict__ partial, int rev) {
  MGD_PDL_ENTRY();
  const long long stride = (long long)gridDim.x * blockDim.x;
  double s0 = 0.0, s1 = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += stride * kMgsU) {
    double2 x[kMgsU], y[kMgsU];
#pragma unroll
    for (int u = 0; u < kMgsU; ++u) {
      const long long k = i + u * stride;
      if (k < n2) {
        const long long e = rev ? n2 - 1 - k : k;
        x[u] = a[e];
        y[u] = b[e];
      } else {
        x[u] = make_double2(0.0, 0.0);
        y[u] = x[u];
      }
    }
#pragma unroll
    for (int u = 0; u < kMgsU; ++u) {
      s0 += x[u].x * y[u].x;
      s1 += x[u].y * y[u].y;
    }
  }
  double s = s0 + s1;
  __shared__ double sh[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) t += sh[k];
    partial[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kThreads) k_mgs_step2(int n2, const double2* __restrict__ vi,
                                                        const double2* __restrict__ vnext, double2* __restrict__ w,
                                                        const double* __restrict__ pin, int nb,
                                                        double* __restrict__ pout, double* __restrict__ hout,
                                                        int rev) {
  MGD_PDL_ENTRY();
  const double h = block_sum_partials(pin, nb);
  if (blockIdx.x == 0 && threadIdx.x == 0) *hout = h;
  const long long stride = (long long)gridDim.x * blockDim.x;
  double s0 = 0.0, s1 = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += stride * kMgsU) {
    double2 ww[kMgsU], a[kMgsU], c[kMgsU];
#pragma unroll
    for (int u = 0; u < kMgsU; ++u) {
      const long long k = i + u * stride;
      if (k < n2) {
        const long long e = rev ? n2 - 1 - k : k;
        ww[u] = w[e];
        a[u] = __ldcs(vi + e);
        c[u] = vnext ? vnext[e] : make_double2(0.0, 0.0);
      }
    }
#pragma unroll
    for (int u = 0; u < kMgsU; ++u) {
      const long long k = i + u * stride;
      if (k < n2) {
        double2 r;
        r.x = ww[u].x - h * a[u].x;
        r.y = ww[u].y - h * a[u].y;
        w[rev ? n2 - 1 - k : k] = r;
        if (vnext) {
          s0 += c[u].x * r.x;
          s1 += c[u].y * r.y;
        } else {
          s0 += r.x * r.x;
          s1 += r.y * r.y;
        }
      }
    }
  }
  double s = s0 + s1;
  __shared__ double sh[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) t += sh[k];
    pout[blockIdx.x] = t;
  }
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

__global__ void k_sum_partials(const double* __restrict__ partial, int nb, double* __restrict__ out) {
  MGD_PDL_ENTRY();
  double r = block_sum_partials(partial, nb);
  if (threadIdx.x == 0) *out = r;
}

// h[0..nv-1] = Gram-Schmidt coefficients of w against V[:, 0..nv-1] (in order),
// w orthogonalised in place, *nrm2 = ||w||^2.  pa / pb: partial buffers of
// kDotBlocks entries each (ping-pong).
void launch_mgs(int n, const double* V, long long ldv, int nv, double* w, double* h, double* nrm2, double* pa,
                double* pb, cudaStream_t s, const std::function<void()>& steps_begin,
                const std::function<void()>& steps_end) {
  int nb = std::min(kDotBlocks, std::max(1, cdiv(n, kThreads)));
  // 16-byte vectors when every basis vector and w start on a 16-byte boundary
  const bool vec = (n % 2 == 0) && (ldv % 2 == 0) && aligned16(V) && aligned16(w);
  const int n2 = n / 2;
  // consecutive passes over the vectors alternate their direction, so each
  // pass starts on the lines the previous one touched last (still in L2):
  // the first dot product runs backwards, step i forwards for even i
  if (vec)
    launch_k(k_dot_partial2, dim3(nb), dim3(kThreads), 0, s, n2, (const double2*)V, (const double2*)w, pa, 1);
  else
    launch_k(k_dot_partial, dim3(nb), dim3(kThreads), 0, s, n, V, w, pa);
  MGD_LAUNCH_CHECK();
  double* pin = pa;
  double* pout = pb;
  if (steps_begin) steps_begin();
  for (int i = 0; i < nv; ++i) {
    const double* vnext = i + 1 < nv ? V + (long long)(i + 1) * ldv : nullptr;
    if (vec)
      launch_k(k_mgs_step2, dim3(nb), dim3(kThreads), 0, s, n2, (const double2*)(V + (long long)i * ldv),
               (const double2*)vnext, (double2*)w, pin, nb, pout, h + i, i & 1);
    else
      launch_k(k_mgs_step, dim3(nb), dim3(kThreads), 0, s, n, V + (long long)i * ldv, vnext, w, pin, nb, pout,
               h + i);
    MGD_LAUNCH_CHECK();
    std::swap(pin, pout);
  }
  if (steps_end) steps_end();
  launch_k(k_sum_partials, dim3(1), dim3(kThreads), 0, s, pin, nb, nrm2);
  MGD_LAUNCH_CHECK();
}

// v = w / ||w||: one reciprocal per block, a multiply per element (FP64
// division is a long instruction sequence on this part)
__global__ void k_scale_by_norm(int n, const double* __restrict__ w, const double* __restrict__ nrm2,
                                double* __restrict__ v) {
  MGD_PDL_ENTRY();
  __shared__ double s_inv;
  if (threadIdx.x == 0) {
    double h = sqrt(*nrm2);
    s_inv = h != 0.0 ? 1.0 / h : 0.0;
  }
  __syncthreads();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = w[i] * s_inv;
}
// ---------------------------------------------------------------- Arnoldi with w resident on chip
// One cooperative grid, one 1024-thread block per SM: block b keeps its slice
// of w in shared memory for the whole modified Gram-Schmidt pass.  Step i
// reads the slice of v_i (its partial <v_i, w> goes to `part`), a grid-wide
// barrier, then every block sums the per-block partials in the same fixed
// order (so all hold the same h_i) and updates w -= h_i v_i in shared memory
// (that second read of v_i comes from L2).  Each basis vector is read once
// from HBM, instead of w being streamed in and out per step.  Ends with
// ||w||^2 and v_out = w / ||w||.
constexpr int kArnThreads = 1024;

__device__ __forceinline__ double arn_block_sum(double v, double* red, double* bc) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kArnThreads / 32; ++k) t += red[k];
    *bc = t;
  }
  __syncthreads();
  return *bc;
}

__global__ void __launch_bounds__(kArnThreads, 1) k_arnoldi_coop(int n, const double* __restrict__ V, long long ldv,
                                                               int nv, const double* __restrict__ w,
                                                               double* __restrict__ h, double* __restrict__ nrm2,
                                                               double* __restrict__ part, double* __restrict__ vout) {
  extern __shared__ double ws[];
  __shared__ double red[kArnThreads / 32];
  __shared__ double bc;
  cg::grid_group grid = cg::this_grid();
  const int nb = gridDim.x, b = blockIdx.x, t = threadIdx.x;
  const long long S = ((long long)n + nb - 1) / nb;
  const long long lo = (long long)b * S;
  const int len = (int)max(0LL, min((long long)n, lo + S) - lo);
  for (int e = t; e < len; e += kArnThreads) ws[e] = w[lo + e];
  // every thread owns the same entries of ws from here on: no block barrier for them
  for (int i = 0; i < nv; ++i) {  // every block runs every step: the grid barriers always match
    const double* vi = V + (long long)i * ldv + lo;
    double d = 0.0;
    for (int e = t; e < len; e += kArnThreads) d += vi[e] * ws[e];
    d = arn_block_sum(d, red, &bc);
    if (t == 0) part[(long long)i * nb + b] = d;
    grid.sync();
    double hi = arn_block_sum(t < nb ? __ldcg(part + (long long)i * nb + t) : 0.0, red, &bc);
    if (b == 0 && t == 0) h[i] = hi;
    for (int e = t; e < len; e += kArnThreads) ws[e] = ws[e] - hi * vi[e];
  }
  double d = 0.0;
  for (int e = t; e < len; e += kArnThreads) d += ws[e] * ws[e];
  d = arn_block_sum(d, red, &bc);
  if (t == 0) part[(long long)nv * nb + b] = d;
  grid.sync();
  double nn = arn_block_sum(t < nb ? __ldcg(part + (long long)nv * nb + t) : 0.0, red, &bc);
  if (b == 0 && t == 0) *nrm2 = nn;
  double hn = sqrt(nn);
  double inv = hn != 0.0 ? 1.0 / hn : 0.0;
  for (int e = t; e < len; e += kArnThreads) vout[lo + e] = ws[e] * inv;
}

// blocks of the cooperative grid (one per SM), or 0 when n does not fit the
// shared memory or the device cannot run the grid
int arnoldi_coop_blocks(int n) {
  int dev = 0, sms = 0, coop = 0, smax = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) ||
      cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) {
    cudaGetLastError();
    return 0;
  }
  if (!coop || sms <= 0 || sms > kArnThreads) return 0;
  long long S = ((long long)n + sms - 1) / sms;
  size_t smem = (size_t)S * sizeof(double);
  size_t stat = (kArnThreads / 32 + 1) * sizeof(double);
  if (smem + stat > (size_t)smax) return 0;
  if (cudaFuncSetAttribute(k_arnoldi_coop, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_arnoldi_coop, kArnThreads, smem) != cudaSuccess ||
      per < 1) {
    cudaGetLastError();
    return 0;
  }
  return sms;
}

void launch_arnoldi_coop(int nb, int n, const double* V, long long ldv, int nv, const double* w, double* h,
                         double* nrm2, double* part, double* vout, cudaStream_t s) {
  long long S = ((long long)n + nb - 1) / nb;
  size_t smem = (size_t)S * sizeof(double);
  void* args[] = {(void*)&n, (void*)&V, (void*)&ldv, (void*)&nv, (void*)&w, (void*)&h, (void*)&nrm2,
                  (void*)&part, (void*)&vout};
  MGD_CUDA(cudaLaunchCooperativeKernel((const void*)k_arnoldi_coop, dim3(nb), dim3(kArnThreads), args, smem, s));
  MGD_LAUNCH_CHECK();
}

// the same on 16-byte vectors, kMgsU pairs per thread and trip (n even, both vectors 16-byte aligned)
__global__ void __launch_bounds__(kThreads) k_scale_by_norm2(int n2, const double2* __restrict__ w,
                                                             const double* __restrict__ nrm2,
                                                             double2* __restrict__ v, int rev) {
  MGD_PDL_ENTRY();
  __shared__ double s_inv;
  if (threadIdx.x == 0) {
    double h = sqrt(*nrm2);
    s_inv = h != 0.0 ? 1.0 / h : 0.0;
  }
  __syncthreads();
  const double r = s_inv;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += stride * kMgsU) {
    double2 a[kMgsU];
#pragma unroll
    for (int u = 0; u < kMgsU; ++u)
      if (i + u * stride < n2) a[u] = w[rev ? n2 - 1 - (i + u * stride) : i + u * stride];
#pragma unroll
    for (int u = 0; u < kMgsU; ++u)
      if (i + u * stride < n2) v[rev ? n2 - 1 - (i + u * stride) : i + u * stride] = make_double2(a[u].x * r, a[u].y * r);
  }
}

void launch_scale_by_norm(int n, const double* w, const double* nrm2, double* v, cudaStream_t s, int rev) {
  if (n % 2 == 0 && aligned16(w) && aligned16(v)) {
    const int n2 = n / 2;
    const int nb = std::min(4 * kDotBlocks, std::max(1, cdiv(n2, kThreads * kMgsU)));
    launch_k(k_scale_by_norm2, dim3(nb), dim3(kThreads), 0, s, n2, (const double2*)w, nrm2, (double2*)v, rev);
  } else {
    launch_k(k_scale_by_norm, dim3(cdiv(n, kThreads)), dim3(kThreads), 0, s, n, w, nrm2, v);
  }
  MGD_LAUNCH_CHECK();
}

__global__ void k_vcomb(int n, const double* __restrict__ Z, long long ldz, int nv, const double* __restrict__ y,
                        double* __restrict__ x) {
  MGD_PDL_ENTRY();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = x[i];
  for (int t = 0; t < nv; ++t) s += y[t] * Z[t * ldz + i];
  x[i] = s;
}
void launch_vcomb(int n, const double* Z, long long ldz, int nv, const double* y, double* x, cudaStream_t s) {
  if (nv <= 0) return;
  launch_k(k_vcomb, dim3(cdiv(n, kThreads)), dim3(kThreads), 0, s, n, Z, ldz, nv, y, x);
  MGD_LAUNCH_CHECK();
}

__global__ void __launch_bounds__(kThreads) k_norm2_partial(int n, const double* __restrict__ x,
                                                            double* __restrict__ partial) {
  MGD_PDL_ENTRY();
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s += x[i] * x[i];
  __shared__ double sh[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) t += sh[k];
    partial[(size_t)blockIdx.x * kMaxV] = t;
  }
}
void launch_norm2(int n, const double* x, double* partial, double* out, cudaStream_t s) {
  int nb = dot_blocks(n);
  launch_k(k_norm2_partial, dim3(nb), dim3(kThreads), 0, s, n, x, partial);
  MGD_LAUNCH_CHECK();
  launch_k(k_reduce_partials, dim3(1), dim3(kThreads), 0, s, partial, nb, 1, out);
  MGD_LAUNCH_CHECK();
}

// PCTL step 2: r_a = v_a - A_a w_a - sum_{b != a} d_ab (.) w_b for every block a
__global__ void k_block_resid(int N, int nc, const int* const* __restrict__ brp, const int* const* __restrict__ bci,
                              const double* const* __restrict__ bv, const double* const* __restrict__ dtab,
                              const IOSlots* __restrict__ io, double* __restrict__ r) {
  MGD_PDL_ENTRY();
  int a = blockIdx.y;
  const double* w = io->z;  // current preconditioner output (the block-relaxed w)
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const int* rp = brp[a];
  const int* ci = bci[a];
  const double* v = bv[a];
  const double* wa = w + (size_t)a * N;
  double s = 0.0;
  for (int p = rp[k]; p < rp[k + 1]; ++p) s += v[p] * wa[ci[p]];
  for (int b = 0; b < nc; ++b) {
    const double* d = dtab[a * nc + b];
    if (b != a && d) s += d[k] * w[(size_t)b * N + k];
  }
  r[(size_t)a * N + k] = io->v[(size_t)a * N + k] - s;
}
void launch_block_resid(int N, int nc, const int* const* brp, const int* const* bci, const double* const* bv,
                        const double* const* dtab, const IOSlots* io, double* r, cudaStream_t s) {
  launch_k(k_block_resid, dim3(dim3(cdiv(N, kThreads), nc)), dim3(kThreads), 0, s, N, nc, brp, bci, bv, dtab, io, r);
  MGD_LAUNCH_CHECK();
}

__global__ void k_saxpy_vec(int n, double a, const double* x, double* y) {
  MGD_PDL_ENTRY();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += a * x[i];
}
void launch_saxpy_vec(int n, double a, const double* x, double* y, cudaStream_t s) {
  launch_k(k_saxpy_vec, dim3(cdiv(n, kThreads)), dim3(kThreads), 0, s, n, a, x, y);
  MGD_LAUNCH_CHECK();
}
__global__ void k_lincomb(int n, double a, const double* x, double b, const double* y, double* out) {
  MGD_PDL_ENTRY();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a * x[i] + b * y[i];
}
void launch_lincomb(int n, double a, const double* x, double b, const double* y, double* out, cudaStream_t s) {
  launch_k(k_lincomb, dim3(cdiv(n, kThreads)), dim3(kThreads), 0, s, n, a, x, b, y, out);
  MGD_LAUNCH_CHECK();
}

}  // namespace mgd

// ---------------------------------------------------------------- device-controlled inverses (Section 3.5)
// Option #3 runs V-cycles on the residual until ||rhs - A x|| <= tol ||rhs||;
// a fixed count > 1 runs the same recurrence a set number of times.  Each
// trip: V-cycle (inactive operators skip it), xacc += x, b = rhs - A xacc with
// partial sums of b^2 in a fixed block order, then one control kernel that
// turns the partial sums into norms, advances the per-operator cycle counts
// and decides which operators stay active.  The host never reads a norm: the
// control kernel also sets the value of the graph's conditional while node.
namespace mgd {

__device__ __forceinline__ void inner_block_partial(double acc, double* out) {
  __shared__ double sh[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) t += sh[k];
    *out = t;
  }
}

// rhs = b, xacc = 0, partial sums of b^2
template <typename T>
__global__ void __launch_bounds__(kThreads) k_inner_begin(const InnerDesc<T>* __restrict__ ds,
                                                          const InnerCtl* __restrict__ ctl) {
  MGD_PDL_ENTRY();
  const InnerDesc<T>* d = ds + blockIdx.y;
  const int n = d->n;
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    T bi = d->b[i];
    d->rhs[i] = bi;
    d->xacc[i] = T(0);
    acc += (double)bi * (double)bi;
  }
  inner_block_partial(acc, ctl->part + (size_t)blockIdx.y * kInnerParts + blockIdx.x);
}

// xacc += x for the active operators
template <typename T>
__global__ void k_inner_update(const InnerDesc<T>* __restrict__ ds) {
  MGD_PDL_ENTRY();
  const InnerDesc<T>* d = ds + blockIdx.y;
  if (*d->active == 0) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < d->n) d->xacc[i] = d->xacc[i] + d->x[i];
}

// b = rhs - A xacc (groups of 4 lanes per row; every thread runs the same
// number of row steps) and partial sums of b^2, for the active operators
template <typename T>
__global__ void __launch_bounds__(kThreads) k_inner_resid(const InnerDesc<T>* __restrict__ ds,
                                                          const InnerCtl* __restrict__ ctl) {
  MGD_PDL_ENTRY();
  const InnerDesc<T>* d = ds + blockIdx.y;
  if (*d->active == 0) return;
  constexpr int TPR = 4;
  const int n = d->n;
  const int lane = threadIdx.x % TPR;
  const long long stride = (long long)gridDim.x * blockDim.x / TPR;
  const long long g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / TPR;
  const long long steps = (n + stride - 1) / stride;
  double acc = 0.0;
  for (long long st = 0; st < steps; ++st) {
    long long row = g + st * stride;
    bool ok = row < n;
    T s = T(0);
    if (ok) {
      int e = d->rp[row + 1];
      for (int p = d->rp[row] + lane; p < e; p += TPR) s += d->v[p] * d->xacc[d->ci[p]];
    }
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (ok && lane == 0) {
      T r = d->rhs[row] - s;
      d->b[row] = r;
      acc += (double)r * (double)r;
    }
  }
  inner_block_partial(acc, ctl->part + (size_t)blockIdx.y * kInnerParts + blockIdx.x);
}

// norms from the partial sums (one warp per operator, fixed order), cycle
// counts, activity; thread 0 publishes "some operator active" to the host
// flag and, under graph replay, to the conditional node
template <typename T>
__global__ void k_inner_ctl(const InnerDesc<T>* __restrict__ ds, int nd, const InnerCtl* __restrict__ ctl, int first,
                            int use_cond, cudaGraphConditionalHandle cond) {
  MGD_PDL_ENTRY();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int mine = 0;
  for (int o = warp; o < nd; o += blockDim.x >> 5) {
    const InnerDesc<T>* d = ds + o;
    double sum = 0.0;
    for (int p = lane; p < kInnerParts; p += 32) sum += ctl->part[(size_t)o * kInnerParts + p];
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, k);
    if (lane == 0) {
      double nr = sqrt(sum);
      int act;
      if (first) {
        ctl->nr0[o] = nr;
        ctl->cycles[o] = 0;
        act = d->accurate ? !(nr <= ctl->tol * nr) : (d->count > 0);
      } else if (*d->active) {
        int c = ++ctl->cycles[o];
        ctl->total[o] += 1;
        act = d->accurate ? (!(nr <= ctl->tol * ctl->nr0[o]) && c < ctl->maxit) : (c < d->count);
      } else {
        act = 0;
      }
      *d->active = act;
      mine |= act;
    }
  }
  int any = __syncthreads_or(mine);
  if (threadIdx.x == 0) {
    int t = first ? 0 : *ctl->trips + 1;
    *ctl->trips = t;
    if (t >= ctl->guard) any = 0;  // hard cap: every operator's own cap is below it
    *ctl->any = any;
    if (use_cond) cudaGraphSetConditional(cond, any ? 1u : 0u);
  }
}

// x = xacc, b = rhs, active = 1
template <typename T>
__global__ void k_inner_end(const InnerDesc<T>* __restrict__ ds) {
  MGD_PDL_ENTRY();
  const InnerDesc<T>* d = ds + blockIdx.y;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < d->n) {
    d->x[i] = d->xacc[i];
    d->b[i] = d->rhs[i];
  }
  if (i == 0) *d->active = 1;
}

template <typename T>
void launch_inner_begin(const InnerDesc<T>* d, int nd, int maxn, const InnerCtl* ctl, cudaStream_t s) {
  (void)maxn;
  launch_k(k_inner_begin<T>, dim3(kInnerParts, nd), dim3(kThreads), 0, s, d, ctl);
  MGD_LAUNCH_CHECK();
}
template <typename T>
void launch_inner_update(const InnerDesc<T>* d, int nd, int maxn, cudaStream_t s) {
  launch_k(k_inner_update<T>, dim3(cdiv(maxn, kThreads), nd), dim3(kThreads), 0, s, d);
  MGD_LAUNCH_CHECK();
}
template <typename T>
void launch_inner_resid(const InnerDesc<T>* d, int nd, int maxn, const InnerCtl* ctl, cudaStream_t s) {
  (void)maxn;
  launch_k(k_inner_resid<T>, dim3(kInnerParts, nd), dim3(kThreads), 0, s, d, ctl);
  MGD_LAUNCH_CHECK();
}
template <typename T>
void launch_inner_ctl(const InnerDesc<T>* d, int nd, const InnerCtl* ctl, int first, int use_cond,
                      cudaGraphConditionalHandle cond, cudaStream_t s) {
  launch_k(k_inner_ctl<T>, dim3(1), dim3(kThreads), 0, s, d, nd, ctl, first, use_cond, cond);
  MGD_LAUNCH_CHECK();
}
template <typename T>
void launch_inner_end(const InnerDesc<T>* d, int nd, int maxn, cudaStream_t s) {
  launch_k(k_inner_end<T>, dim3(cdiv(std::max(maxn, 1), kThreads), nd), dim3(kThreads), 0, s, d);
  MGD_LAUNCH_CHECK();
}

#define MGD_INNER_INST(T)                                                                                      \
  template void launch_inner_begin<T>(const InnerDesc<T>*, int, int, const InnerCtl*, cudaStream_t);          \
  template void launch_inner_update<T>(const InnerDesc<T>*, int, int, cudaStream_t);                          \
  template void launch_inner_resid<T>(const InnerDesc<T>*, int, int, const InnerCtl*, cudaStream_t);          \
  template void launch_inner_ctl<T>(const InnerDesc<T>*, int, const InnerCtl*, int, int,                      \
                                    cudaGraphConditionalHandle, cudaStream_t);                                 \
  template void launch_inner_end<T>(const InnerDesc<T>*, int, int, cudaStream_t);
MGD_INNER_INST(double)
MGD_INNER_INST(float)
#undef MGD_INNER_INST

}  // namespace mgd
