// solve_kernels.cu -- device kernels of the solve phase: the V(1,1) cycle
// (Section 3.1) on every level, the block-level updates of the block
// preconditioners (Sections 3.3-3.4), and the FGMRES vector work.
//
// All of these are HBM-bound sparse or streaming kernels.  Sparse rows are
// read either from a sliced ELL layout (32-row slices stored column-major, so
// a warp reads 32 consecutive values per step: fully coalesced) or from CSR
// with TPR threads per row (warp-shuffle reduction).  The format is chosen per
// level at setup by timing.  Every kernel of one V-cycle phase runs over all
// subsystems of a batch at once: blockIdx.y selects the subsystem.
#include "mgd_internal.cuh"

namespace mgd {

template <int FMT>
struct FmtTraits {
  static constexpr int tpr = 1;
};
template <> struct FmtTraits<FMT_CSR2> { static constexpr int tpr = 2; };
template <> struct FmtTraits<FMT_CSR4> { static constexpr int tpr = 4; };
template <> struct FmtTraits<FMT_CSR8> { static constexpr int tpr = 8; };
template <> struct FmtTraits<FMT_CSR16> { static constexpr int tpr = 16; };
template <> struct FmtTraits<FMT_CSR32> { static constexpr int tpr = 32; };

// x accessors
template <typename T>
struct XPlain {
  const T* x;
  __device__ __forceinline__ T operator()(int j) const { return __ldg(x + j); }
};
template <typename T>
struct XScaled {  // x_j = dinv_j * b_j (the zero-guess Jacobi iterate)
  const T* d;
  const T* b;
  __device__ __forceinline__ T operator()(int j) const { return __ldg(d + j) * __ldg(b + j); }
};

// Row dot product sum_p a_ip x(ci_p).  Every lane of the calling warp must
// reach this function (shuffles); lanes whose row is out of range pass
// valid = false and get 0.
template <typename T, int FMT, class XF>
__device__ __forceinline__ T row_dot(int row, int lane, bool valid, const int* __restrict__ rp,
                                     const int* __restrict__ ci, const T* __restrict__ v,
                                     const int* __restrict__ sptr, const int* __restrict__ sci,
                                     const T* __restrict__ sv, const XF& xf) {
  T s = T(0);
  if (FMT == FMT_SELL) {
    if (valid) {
      int sl = row >> 5, ln = row & 31;
      int base = __ldg(sptr + sl);
      int width = (__ldg(sptr + sl + 1) - base) >> 5;
      const int* c = sci + base + ln;
      const T* a = sv + base + ln;
#pragma unroll 4
      for (int j = 0; j < width; ++j) s += __ldg(a + 32 * j) * xf(__ldg(c + 32 * j));
    }
  } else {
    constexpr int TPR = FmtTraits<FMT>::tpr;
    if (valid) {
      int b = __ldg(rp + row), e = __ldg(rp + row + 1);
#pragma unroll 2
      for (int p = b + lane; p < e; p += TPR) s += __ldg(v + p) * xf(__ldg(ci + p));
    }
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;
}

// ---------------------------------------------------------------- V-cycle phases
// PRE: xt = D^-1 b (zero initial guess), r = b - A xt = b - (A D^-1) b, using
// the column-scaled copy of A so that each nonzero costs one multiply-add
template <typename T, int FMT>
__global__ void __launch_bounds__(kThreads) k_pre(const LDesc<T>* __restrict__ descs) {
  const LDesc<T>* d = descs + blockIdx.y;
  constexpr int TPR = FmtTraits<FMT>::tpr;
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  int row = g / TPR, lane = g % TPR;
  int n = d->n;
  if (((g & ~31) / TPR) >= n) return;  // the whole warp is past the last row (TPR divides 32)
  bool valid = row < n;
  const T* b = d->b;
  XPlain<T> xf{b};
  T s = row_dot<T, FMT>(row, lane, valid, d->rp, d->ci, d->vpre, d->sptr, d->sci, d->svpre, xf);
  if (valid && lane == 0) {
    T bi = b[row];
    d->xt[row] = d->dinv[row] * bi;
    d->r[row] = bi - s;
  }
}

// POST: x = xt + D^-1 (b - A xt)
template <typename T, int FMT>
__global__ void __launch_bounds__(kThreads) k_post(const LDesc<T>* __restrict__ descs) {
  const LDesc<T>* d = descs + blockIdx.y;
  constexpr int TPR = FmtTraits<FMT>::tpr;
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  int row = g / TPR, lane = g % TPR;
  int n = d->n;
  if (((g & ~31LL) / TPR) >= n) return;
  bool valid = row < n;
  XPlain<T> xf{d->xt};
  T s = row_dot<T, FMT>(row, lane, valid, d->rp, d->ci, d->v, d->sptr, d->sci, d->sv, xf);
  if (valid && lane == 0) d->x[row] = d->xt[row] + d->dinv[row] * (d->b[row] - s);
}

// RESTRICT: bc = R r ; PROLONG: xt += P xc  (CSR, TPR threads per row)
template <typename T, int FMT>
__global__ void __launch_bounds__(kThreads) k_restrict(const LDesc<T>* __restrict__ descs) {
  const LDesc<T>* d = descs + blockIdx.y;
  constexpr int TPR = FmtTraits<FMT>::tpr;
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  int row = g / TPR, lane = g % TPR;
  int n = d->nc;
  if (((g & ~31LL) / TPR) >= n) return;
  bool valid = row < n;
  XPlain<T> xf{d->r};
  T s = row_dot<T, FMT>(row, lane, valid, d->rrp, d->rci, d->rv, nullptr, nullptr, nullptr, xf);
  if (valid && lane == 0) d->bc[row] = s;
}

template <typename T, int FMT>
__global__ void __launch_bounds__(kThreads) k_prolong(const LDesc<T>* __restrict__ descs) {
  const LDesc<T>* d = descs + blockIdx.y;
  constexpr int TPR = FmtTraits<FMT>::tpr;
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  int row = g / TPR, lane = g % TPR;
  int n = d->n;
  if (((g & ~31LL) / TPR) >= n) return;
  bool valid = row < n;
  XPlain<T> xf{d->xc};
  T s = row_dot<T, FMT>(row, lane, valid, d->prp, d->pci, d->pv, nullptr, nullptr, nullptr, xf);
  if (valid && lane == 0) d->xt[row] += s;
}

// stalled coarsest level, first l1-Jacobi sweep from zero: xt = D^-1 b
template <typename T>
__global__ void k_jac1(const LDesc<T>* __restrict__ descs) {
  const LDesc<T>* d = descs + blockIdx.y;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < d->n) d->xt[i] = d->dinv[i] * d->b[i];
}

// coarsest level: x = A_L^{-1} b with the dense FP64 inverse (one CTA per subsystem)
template <typename T>
__global__ void k_coarse(const LDesc<T>* __restrict__ descs) {
  const LDesc<T>* d = descs + blockIdx.y;
  extern __shared__ double sb[];
  int n = d->cn;
  for (int j = threadIdx.x; j < n; j += blockDim.x) sb[j] = (double)d->b[j];
  __syncthreads();
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = warp; i < n; i += nw) {
    const double* row = d->cinv + (size_t)i * n;
    double s = 0.0;
    for (int j = lane; j < n; j += 32) s += row[j] * sb[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) d->x[i] = (T)s;
  }
}

#define MGD_DISPATCH_FMT(K, fmt, maxrows, ny, s, descs)                                        \
  do {                                                                                         \
    auto g_ = [&](int tpr) { return dim3(cdiv((long long)(maxrows) * tpr + 32, kThreads), (ny)); }; \
    switch (fmt) {                                                                             \
      case FMT_SELL: K<T, FMT_SELL><<<g_(1), kThreads, 0, s>>>(descs); break;                  \
      case FMT_CSR1: K<T, FMT_CSR1><<<g_(1), kThreads, 0, s>>>(descs); break;                  \
      case FMT_CSR2: K<T, FMT_CSR2><<<g_(2), kThreads, 0, s>>>(descs); break;                  \
      case FMT_CSR4: K<T, FMT_CSR4><<<g_(4), kThreads, 0, s>>>(descs); break;                  \
      case FMT_CSR8: K<T, FMT_CSR8><<<g_(8), kThreads, 0, s>>>(descs); break;                  \
      case FMT_CSR16: K<T, FMT_CSR16><<<g_(16), kThreads, 0, s>>>(descs); break;               \
      default: K<T, FMT_CSR32><<<g_(32), kThreads, 0, s>>>(descs); break;                      \
    }                                                                                          \
  } while (0)

template <typename T>
void launch_phase(int phase, int fmtA, int fmtRP, const LDesc<T>* d_descs, int ndesc, int maxrows, cudaStream_t s) {
  if (ndesc <= 0 || maxrows <= 0) return;
  int rp = fmtRP == FMT_SELL ? FMT_CSR1 : fmtRP;
  switch (phase) {
    case PH_PRE: MGD_DISPATCH_FMT(k_pre, fmtA, maxrows, ndesc, s, d_descs); break;
    case PH_POST: MGD_DISPATCH_FMT(k_post, fmtA, maxrows, ndesc, s, d_descs); break;
    case PH_RESTRICT: MGD_DISPATCH_FMT(k_restrict, rp, maxrows, ndesc, s, d_descs); break;
    case PH_PROLONG: MGD_DISPATCH_FMT(k_prolong, rp, maxrows, ndesc, s, d_descs); break;
    case PH_JAC1: k_jac1<T><<<dim3(cdiv(maxrows, kThreads), ndesc), kThreads, 0, s>>>(d_descs); break;
    case PH_COARSE:
      k_coarse<T><<<dim3(1, ndesc), kThreads, sizeof(double) * maxrows, s>>>(d_descs);
      break;
  }
  MGD_LAUNCH_CHECK();
}

template void launch_phase<double>(int, int, int, const LDesc<double>*, int, int, cudaStream_t);
template void launch_phase<float>(int, int, int, const LDesc<float>*, int, int, cudaStream_t);

// ---------------------------------------------------------------- block-level updates
__device__ __forceinline__ double* resolve(const PRef& r, const IOSlots* io) {
  if (r.slot == 0) return r.abs;
  if (r.slot == 1) return const_cast<double*>(io->v) + r.off;
  return io->z + r.off;
}

// dst = (T)(a + sum_t s_t d_t (.) w_t)
template <typename T>
__global__ void k_produce(const ProduceDesc<T>* __restrict__ ds, int N, const IOSlots* __restrict__ io) {
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
  d->dst[k] = (T)acc;
}

// dst = base + s * x
template <typename T>
__global__ void k_consume(const ConsumeDesc<T>* __restrict__ ds, int N, const IOSlots* __restrict__ io) {
  const ConsumeDesc<T>* d = ds + blockIdx.y;
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  double* dst = resolve(d->dst, io);
  const double* base = resolve(d->base, io);
  double val = d->s * (double)d->x[k];
  dst[k] = base ? base[k] + val : val;
}

template <typename T>
__global__ void k_jacobi(const JacDesc<T>* __restrict__ ds, int N) {
  const JacDesc<T>* d = ds + blockIdx.y;
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < N) d->x[k] = d->dinv[k] * d->b[k];
}

template <typename T>
void launch_produce(const ProduceDesc<T>* d, int nd, int N, const IOSlots* io, cudaStream_t s) {
  if (nd <= 0) return;
  k_produce<T><<<dim3(cdiv(N, kThreads), nd), kThreads, 0, s>>>(d, N, io);
  MGD_LAUNCH_CHECK();
}
template <typename T>
void launch_consume(const ConsumeDesc<T>* d, int nd, int N, const IOSlots* io, cudaStream_t s) {
  if (nd <= 0) return;
  k_consume<T><<<dim3(cdiv(N, kThreads), nd), kThreads, 0, s>>>(d, N, io);
  MGD_LAUNCH_CHECK();
}
template <typename T>
void launch_jacobi(const JacDesc<T>* d, int nd, int N, cudaStream_t s) {
  if (nd <= 0) return;
  k_jacobi<T><<<dim3(cdiv(N, kThreads), nd), kThreads, 0, s>>>(d, N);
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
  constexpr int TPR = FmtTraits<FMT>::tpr;
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int row = (int)(g / TPR), lane = (int)(g % TPR);
  if (((g & ~31LL) / TPR) >= n) return;
  bool valid = row < n;
  XPlain<T> xf{x};
  T s = row_dot<T, FMT>(row, lane, valid, rp, ci, v, sptr, sci, sv, xf);
  if (valid && lane == 0) y[row] = MODE ? b[row] - s : s;
}

template <typename T, int MODE>
static void spmv_dispatch(int fmt, int n, const int* rp, const int* ci, const T* v, const int* sptr,
                          const int* sci, const T* sv, const T* b, const T* x, T* y, cudaStream_t s) {
  if (n <= 0) return;
  if (fmt == FMT_SELL && !sptr) fmt = FMT_CSR4;
  auto g = [&](int tpr) { return cdiv((long long)n * tpr + 32, kThreads); };
  switch (fmt) {
    case FMT_SELL: k_spmv<T, FMT_SELL, MODE><<<g(1), kThreads, 0, s>>>(n, rp, ci, v, sptr, sci, sv, b, x, y); break;
    case FMT_CSR1: k_spmv<T, FMT_CSR1, MODE><<<g(1), kThreads, 0, s>>>(n, rp, ci, v, sptr, sci, sv, b, x, y); break;
    case FMT_CSR2: k_spmv<T, FMT_CSR2, MODE><<<g(2), kThreads, 0, s>>>(n, rp, ci, v, sptr, sci, sv, b, x, y); break;
    case FMT_CSR4: k_spmv<T, FMT_CSR4, MODE><<<g(4), kThreads, 0, s>>>(n, rp, ci, v, sptr, sci, sv, b, x, y); break;
    case FMT_CSR8: k_spmv<T, FMT_CSR8, MODE><<<g(8), kThreads, 0, s>>>(n, rp, ci, v, sptr, sci, sv, b, x, y); break;
    case FMT_CSR16:
      k_spmv<T, FMT_CSR16, MODE><<<g(16), kThreads, 0, s>>>(n, rp, ci, v, sptr, sci, sv, b, x, y);
      break;
    default: k_spmv<T, FMT_CSR32, MODE><<<g(32), kThreads, 0, s>>>(n, rp, ci, v, sptr, sci, sv, b, x, y); break;
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
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += x[i];
}
template <typename T>
void launch_axpy(int n, T* y, const T* x, cudaStream_t s) {
  if (n <= 0) return;
  k_axpy<T><<<cdiv(n, kThreads), kThreads, 0, s>>>(n, y, x);
  MGD_LAUNCH_CHECK();
}
template void launch_axpy<double>(int, double*, const double*, cudaStream_t);
template void launch_axpy<float>(int, float*, const float*, cudaStream_t);

__global__ void k_set_io(IOSlots* io, const double* v, double* z) {
  io->v = v;
  io->z = z;
}
void launch_set_io(IOSlots* io, const double* v, double* z, cudaStream_t s) {
  k_set_io<<<1, 1, 0, s>>>(io, v, z);
  MGD_LAUNCH_CHECK();
}

__global__ void k_cast_df(int n, const double* a, float* b) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}
__global__ void k_cast_fd(int n, const float* a, double* b) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}
__global__ void k_copy(int n, const double* a, double* b) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = a[i];
}
void launch_cast_f64_f32(int n, const double* a, float* b, cudaStream_t s) {
  if (n <= 0) return;
  k_cast_df<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, a, b);
  MGD_LAUNCH_CHECK();
}
void launch_cast_f32_f64(int n, const float* a, double* b, cudaStream_t s) {
  if (n <= 0) return;
  k_cast_fd<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, a, b);
  MGD_LAUNCH_CHECK();
}
void launch_copy_f64(int n, const double* a, double* b, cudaStream_t s) {
  if (n <= 0) return;
  k_copy<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, a, b);
  MGD_LAUNCH_CHECK();
}

// ---------------------------------------------------------------- Arnoldi (FP64)
constexpr int kMaxV = 32;

// Classical Gram-Schmidt with a selective second pass (Daniel, Gragg, Kaufman,
// Stewart 1976): the second projection runs only when the first one removed
// more than half of ||w||^2, a test the kernels read from device memory
// (cond_after < 0.5 cond_before), so no host round trip is needed.
__device__ __forceinline__ bool second_pass_needed(const double* after, const double* before) {
  return !after || after[0] < 0.5 * before[0];
}

// partial[b * kMaxV + t] = sum over this block's elements of V_t(i) w(i); with
// selfdot, slot nv gets w.w.  Skipped (zeros) when cond says no second pass.
template <int NV>
__global__ void __launch_bounds__(kThreads) k_mdot(int n, const double* __restrict__ V, long long ldv, int nv,
                                                   const double* __restrict__ w, double* __restrict__ partial,
                                                   int selfdot, const double* __restrict__ cond_after,
                                                   const double* __restrict__ cond_before) {
  if (!second_pass_needed(cond_after, cond_before)) {
    for (int t = threadIdx.x; t < NV; t += blockDim.x) partial[(size_t)blockIdx.x * kMaxV + t] = 0.0;
    return;
  }
  double acc[NV];
#pragma unroll
  for (int t = 0; t < NV; ++t) acc[t] = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double wi = w[i];
#pragma unroll
    for (int t = 0; t < NV; ++t) {
      if (t < nv) acc[t] += V[t * ldv + i] * wi;
      else if (t == nv && selfdot) acc[t] += wi * wi;
    }
  }
  __shared__ double sh[kThreads / 32][NV];
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int t = 0; t < NV; ++t) {
    double s = acc[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) sh[warp][t] = s;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < NV; t += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) s += sh[k][t];
    partial[(size_t)blockIdx.x * kMaxV + t] = s;
  }
}

// out[t] = sum_b partial[b * kMaxV + t]  (fixed order: deterministic)
__global__ void k_reduce_partials(const double* __restrict__ partial, int nblocks, int nv, double* __restrict__ out) {
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

void launch_mdot(int n, const double* V, long long ldv, int nv, const double* w, double* partial, double* out,
                 cudaStream_t s, int selfdot, const double* cond_after, const double* cond_before) {
  int nb = dot_blocks(n);
  int nt = nv + (selfdot ? 1 : 0);
  if (nt <= 4) k_mdot<4><<<nb, kThreads, 0, s>>>(n, V, ldv, nv, w, partial, selfdot, cond_after, cond_before);
  else if (nt <= 8) k_mdot<8><<<nb, kThreads, 0, s>>>(n, V, ldv, nv, w, partial, selfdot, cond_after, cond_before);
  else if (nt <= 16) k_mdot<16><<<nb, kThreads, 0, s>>>(n, V, ldv, nv, w, partial, selfdot, cond_after, cond_before);
  else k_mdot<32><<<nb, kThreads, 0, s>>>(n, V, ldv, nv, w, partial, selfdot, cond_after, cond_before);
  MGD_LAUNCH_CHECK();
  k_reduce_partials<<<nt, kThreads, 0, s>>>(partial, nb, nt, out);
  MGD_LAUNCH_CHECK();
}

// w -= sum_t h_t V_t, and partial norms of the new w.  Skipped when cond says
// no second pass: then the norm partials carry the first pass's ||w||^2.
template <int NV>
__global__ void __launch_bounds__(kThreads) k_vupdate(int n, const double* __restrict__ V, long long ldv, int nv,
                                                      const double* __restrict__ h, double* __restrict__ w,
                                                      double* __restrict__ partial, const double* __restrict__ cond_after,
                                                      const double* __restrict__ cond_before) {
  if (!second_pass_needed(cond_after, cond_before)) {
    if (threadIdx.x == 0) partial[(size_t)blockIdx.x * kMaxV] = blockIdx.x == 0 ? cond_after[0] : 0.0;
    return;
  }
  __shared__ double sh_h[NV];
  for (int t = threadIdx.x; t < NV; t += blockDim.x) sh_h[t] = t < nv ? h[t] : 0.0;
  __syncthreads();
  double nrm = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double wi = w[i];
#pragma unroll
    for (int t = 0; t < NV; ++t)
      if (t < nv) wi -= sh_h[t] * V[t * ldv + i];
    w[i] = wi;
    nrm += wi * wi;
  }
  __shared__ double sh[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = nrm;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) s += sh[k];
    partial[(size_t)blockIdx.x * kMaxV] = s;
  }
}

void launch_vupdate(int n, const double* V, long long ldv, int nv, const double* h, double* w, double* partial,
                    double* nrm2, cudaStream_t s, const double* cond_after, const double* cond_before) {
  int nb = dot_blocks(n);
  if (nv <= 4) k_vupdate<4><<<nb, kThreads, 0, s>>>(n, V, ldv, nv, h, w, partial, cond_after, cond_before);
  else if (nv <= 8) k_vupdate<8><<<nb, kThreads, 0, s>>>(n, V, ldv, nv, h, w, partial, cond_after, cond_before);
  else if (nv <= 16) k_vupdate<16><<<nb, kThreads, 0, s>>>(n, V, ldv, nv, h, w, partial, cond_after, cond_before);
  else k_vupdate<32><<<nb, kThreads, 0, s>>>(n, V, ldv, nv, h, w, partial, cond_after, cond_before);
  MGD_LAUNCH_CHECK();
  k_reduce_partials<<<1, kThreads, 0, s>>>(partial, nb, 1, nrm2);
  MGD_LAUNCH_CHECK();
}

// v = w / ||w||: one reciprocal per block, a multiply per element (FP64
// division is a long instruction sequence on this part)
__global__ void k_scale_by_norm(int n, const double* __restrict__ w, const double* __restrict__ nrm2,
                                double* __restrict__ v) {
  __shared__ double s_inv;
  if (threadIdx.x == 0) {
    double h = sqrt(*nrm2);
    s_inv = h != 0.0 ? 1.0 / h : 0.0;
  }
  __syncthreads();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = w[i] * s_inv;
}
void launch_scale_by_norm(int n, const double* w, const double* nrm2, double* v, cudaStream_t s) {
  k_scale_by_norm<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, w, nrm2, v);
  MGD_LAUNCH_CHECK();
}

__global__ void k_vcomb(int n, const double* __restrict__ Z, long long ldz, int nv, const double* __restrict__ y,
                        double* __restrict__ x) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = x[i];
  for (int t = 0; t < nv; ++t) s += y[t] * Z[t * ldz + i];
  x[i] = s;
}
void launch_vcomb(int n, const double* Z, long long ldz, int nv, const double* y, double* x, cudaStream_t s) {
  if (nv <= 0) return;
  k_vcomb<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, Z, ldz, nv, y, x);
  MGD_LAUNCH_CHECK();
}

__global__ void __launch_bounds__(kThreads) k_norm2_partial(int n, const double* __restrict__ x,
                                                            double* __restrict__ partial) {
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
  k_norm2_partial<<<nb, kThreads, 0, s>>>(n, x, partial);
  MGD_LAUNCH_CHECK();
  k_reduce_partials<<<1, kThreads, 0, s>>>(partial, nb, 1, out);
  MGD_LAUNCH_CHECK();
}

// PCTL step 2: r_a = v_a - A_a w_a - sum_{b != a} d_ab (.) w_b for every block a
__global__ void k_block_resid(int N, int nc, const int* const* __restrict__ brp, const int* const* __restrict__ bci,
                              const double* const* __restrict__ bv, const double* const* __restrict__ dtab,
                              const IOSlots* __restrict__ io, double* __restrict__ r) {
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
  k_block_resid<<<dim3(cdiv(N, kThreads), nc), kThreads, 0, s>>>(N, nc, brp, bci, bv, dtab, io, r);
  MGD_LAUNCH_CHECK();
}

__global__ void k_saxpy_vec(int n, double a, const double* x, double* y) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += a * x[i];
}
void launch_saxpy_vec(int n, double a, const double* x, double* y, cudaStream_t s) {
  k_saxpy_vec<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, a, x, y);
  MGD_LAUNCH_CHECK();
}
__global__ void k_lincomb(int n, double a, const double* x, double b, const double* y, double* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a * x[i] + b * y[i];
}
void launch_lincomb(int n, double a, const double* x, double b, const double* y, double* out, cudaStream_t s) {
  k_lincomb<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, a, x, b, y, out);
  MGD_LAUNCH_CHECK();
}

}  // namespace mgd
