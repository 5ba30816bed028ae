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

}  // namespace mgd
