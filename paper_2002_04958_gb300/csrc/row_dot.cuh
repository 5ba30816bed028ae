// row_dot.cuh -- sparse row dot products shared by the V-cycle and SpMV kernels.
#pragma once
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

// Two-phase row dot product for kernels launched with programmatic dependent
// launch: row_load fetches the row's extent and its first PRE entries (column
// index and value) per lane -- operator data, which no predecessor kernel of
// the solve writes -- so those dependent loads overlap the previous kernel;
// row_finish (after the dependency wait) gathers x and completes the row.
// The products are accumulated in the same order as row_dot.
template <typename T, int PRE>
struct RowPre {
  int p, e;  // CSR: next entry of this lane after the preloaded ones, row end; SELL: base, width
  int ln;
  int c[PRE];
  T a[PRE];
};

template <typename T, int FMT, int PRE>
__device__ __forceinline__ void row_load(RowPre<T, PRE>& R, int row, int lane, bool valid, const int* __restrict__ rp,
                                         const int* __restrict__ ci, const T* __restrict__ v,
                                         const int* __restrict__ sptr, const int* __restrict__ sci,
                                         const T* __restrict__ sv) {
  R.p = 0;
  R.e = 0;
  R.ln = 0;
  if (!valid) return;
  if (FMT == FMT_SELL) {
    int sl = row >> 5;
    R.ln = row & 31;
    R.p = __ldg(sptr + sl);
    R.e = (__ldg(sptr + sl + 1) - R.p) >> 5;  // width
#pragma unroll
    for (int k = 0; k < PRE; ++k)
      if (k < R.e) {
        R.c[k] = __ldg(sci + R.p + 32 * k + R.ln);
        R.a[k] = __ldg(sv + R.p + 32 * k + R.ln);
      }
  } else {
    constexpr int TPR = FmtTraits<FMT>::tpr;
    int b = __ldg(rp + row);
    R.e = __ldg(rp + row + 1);
#pragma unroll
    for (int k = 0; k < PRE; ++k) {
      int q = b + lane + k * TPR;
      if (q < R.e) {
        R.c[k] = __ldg(ci + q);
        R.a[k] = __ldg(v + q);
      }
    }
    R.p = b + lane + PRE * TPR;
  }
}

template <typename T, int FMT, int PRE, class XF>
__device__ __forceinline__ T row_finish(const RowPre<T, PRE>& R, bool valid, const int* __restrict__ ci,
                                        const T* __restrict__ v, const int* __restrict__ sci,
                                        const T* __restrict__ sv, const XF& xf) {
  T s = T(0);
  if (FMT == FMT_SELL) {
    if (valid) {
#pragma unroll
      for (int k = 0; k < PRE; ++k)
        if (k < R.e) s += R.a[k] * xf(R.c[k]);
      const int* c = sci + R.p + R.ln;
      const T* a = sv + R.p + R.ln;
      for (int j = PRE; j < R.e; ++j) s += __ldg(a + 32 * j) * xf(__ldg(c + 32 * j));
    }
  } else {
    constexpr int TPR = FmtTraits<FMT>::tpr;
    if (valid) {
      const int first = R.p - PRE * TPR;
#pragma unroll
      for (int k = 0; k < PRE; ++k)
        if (first + k * TPR < R.e) s += R.a[k] * xf(R.c[k]);
      for (int q = R.p; q < R.e; q += TPR) s += __ldg(v + q) * xf(__ldg(ci + q));
    }
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;
}

}  // namespace mgd
