// vcycle_kernels.cu -- the V(1,1) cycle phases (Section 3.1) on every level:
// pre-smoothing + residual, restriction, prolongation, post-smoothing, and the
// coarsest-level solve.
//
// HBM-bound sparse kernels.  Rows are read either from a sliced ELL layout
// (32-row slices stored column-major, so a warp reads 32 consecutive values
// per step: fully coalesced) or from CSR with TPR threads per row
// (warp-shuffle reduction); the layout is chosen per level at setup by timing.
// Every launch serves all subsystems of a batch: blockIdx.y selects the
// subsystem's level descriptor.
#include "mgd_internal.cuh"
#include "row_dot.cuh"

#include <cooperative_groups.h>

namespace mgd {

// ---------------------------------------------------------------- V-cycle phases
// Each phase kernel loads its rows' operator entries (and the smoother
// diagonal) before the dependency wait -- setup-time data -- and gathers the
// vector its predecessor wrote only after it.
// threads per CTA of the per-level V-cycle kernels
#ifndef MGD_VTHREADS
#define MGD_VTHREADS 256
#endif
constexpr int kVThreads = MGD_VTHREADS;
#ifndef MGD_KPRE
#define MGD_KPRE 5
#endif
constexpr int kPre = MGD_KPRE;  // entries per lane loaded before the wait

// PRE: xt = D^-1 b (zero initial guess), r = b - A xt = b - (A D^-1) b, using
// the column-scaled copy of A so that each nonzero costs one multiply-add
template <typename T, int FMT>
__global__ void __launch_bounds__(kVThreads) k_pre(const LDesc<T>* __restrict__ descs) {
  MGD_PDL_TRIGGER();
  const LDesc<T>* d = descs + blockIdx.y;
  constexpr int TPR = FmtTraits<FMT>::tpr;
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  int row = g / TPR, lane = g % TPR;
  int n = d->n;
  if (((g & ~31) / TPR) >= n) return;  // the whole warp is past the last row (TPR divides 32)
  bool valid = row < n;
  RowPre<T, kPre> R;
  row_load<T, FMT, kPre>(R, row, lane, valid, d->rp, d->ci, d->vpre, d->sptr, d->sci, d->svpre);
  T di = valid && lane == 0 ? d->dinv[row] : T(0);
  MGD_PDL_WAIT();
  MGD_SKIP_INACTIVE(d);
  const T* b = d->b;
  XPlain<T> xf{b};
  T s = row_finish<T, FMT, kPre>(R, valid, d->ci, d->vpre, d->sci, d->svpre, xf);
  if (valid && lane == 0) {
    T bi = b[row];
    d->xt[row] = di * bi;
    d->r[row] = bi - s;
  }
}

// POST: x = xt + D^-1 (b - A xt)
template <typename T, int FMT>
__global__ void __launch_bounds__(kVThreads) k_post(const LDesc<T>* __restrict__ descs) {
  MGD_PDL_TRIGGER();
  const LDesc<T>* d = descs + blockIdx.y;
  constexpr int TPR = FmtTraits<FMT>::tpr;
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  int row = g / TPR, lane = g % TPR;
  int n = d->n;
  if (((g & ~31LL) / TPR) >= n) return;
  bool valid = row < n;
  RowPre<T, kPre> R;
  row_load<T, FMT, kPre>(R, row, lane, valid, d->rp, d->ci, d->v, d->sptr, d->sci, d->sv);
  T di = valid && lane == 0 ? d->dinv[row] : T(0);
  MGD_PDL_WAIT();
  MGD_SKIP_INACTIVE(d);
  XPlain<T> xf{d->xt};
  T s = row_finish<T, FMT, kPre>(R, valid, d->ci, d->v, d->sci, d->sv, xf);
  if (valid && lane == 0) d->x[row] = d->xt[row] + di * (d->b[row] - s);
}

// Multi-slice forms of PRE and POST (FMT_SELL2, FMT_SELL4): each thread smooths
// the same lane of K adjacent 32-row slices, so K rows' loads are in flight per
// thread (the row sums are those of the SELL kernels)
template <typename T, int K>
__global__ void __launch_bounds__(kVThreads) k_pre_sk(const LDesc<T>* __restrict__ descs) {
  MGD_PDL_TRIGGER();
  const LDesc<T>* d = descs + blockIdx.y;
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  int w = g >> 5, lane = g & 31;
  int n = d->n;
  if (w * 32 * K >= n) return;  // the whole warp is past the last row
  RowPre<T, kPre> R[K];
  T di[K];
#pragma unroll
  for (int q = 0; q < K; ++q) {
    int r = (w * K + q) * 32 + lane;
    row_load<T, FMT_SELL, kPre>(R[q], r, 0, r < n, nullptr, nullptr, nullptr, d->sptr, d->sci, d->svpre);
    di[q] = r < n ? d->dinv[r] : T(0);
  }
  MGD_PDL_WAIT();
  MGD_SKIP_INACTIVE(d);
  const T* b = d->b;
  XPlain<T> xf{b};
#pragma unroll
  for (int q = 0; q < K; ++q) {
    int r = (w * K + q) * 32 + lane;
    T s = row_finish<T, FMT_SELL, kPre>(R[q], r < n, nullptr, nullptr, d->sci, d->svpre, xf);
    if (r < n) {
      T bi = b[r];
      d->xt[r] = di[q] * bi;
      d->r[r] = bi - s;
    }
  }
}

template <typename T, int K>
__global__ void __launch_bounds__(kVThreads) k_post_sk(const LDesc<T>* __restrict__ descs) {
  MGD_PDL_TRIGGER();
  const LDesc<T>* d = descs + blockIdx.y;
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  int w = g >> 5, lane = g & 31;
  int n = d->n;
  if (w * 32 * K >= n) return;
  RowPre<T, kPre> R[K];
  T di[K];
#pragma unroll
  for (int q = 0; q < K; ++q) {
    int r = (w * K + q) * 32 + lane;
    row_load<T, FMT_SELL, kPre>(R[q], r, 0, r < n, nullptr, nullptr, nullptr, d->sptr, d->sci, d->sv);
    di[q] = r < n ? d->dinv[r] : T(0);
  }
  MGD_PDL_WAIT();
  MGD_SKIP_INACTIVE(d);
  XPlain<T> xf{d->xt};
#pragma unroll
  for (int q = 0; q < K; ++q) {
    int r = (w * K + q) * 32 + lane;
    T s = row_finish<T, FMT_SELL, kPre>(R[q], r < n, nullptr, nullptr, d->sci, d->sv, xf);
    if (r < n) d->x[r] = d->xt[r] + di[q] * (d->b[r] - s);
  }
}

// RESTRICT: bc = R r ; PROLONG: xt += P xc  (CSR, TPR threads per row)
template <typename T, int FMT>
__global__ void __launch_bounds__(kVThreads) k_restrict(const LDesc<T>* __restrict__ descs) {
  MGD_PDL_TRIGGER();
  const LDesc<T>* d = descs + blockIdx.y;
  constexpr int TPR = FmtTraits<FMT>::tpr;
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  int row = g / TPR, lane = g % TPR;
  int n = d->nc;
  if (((g & ~31LL) / TPR) >= n) return;
  bool valid = row < n;
  RowPre<T, kPre> R;
  row_load<T, FMT, kPre>(R, row, lane, valid, d->rrp, d->rci, d->rv, nullptr, nullptr, nullptr);
  MGD_PDL_WAIT();
  MGD_SKIP_INACTIVE(d);
  XPlain<T> xf{d->r};
  T s = row_finish<T, FMT, kPre>(R, valid, d->rci, d->rv, nullptr, nullptr, xf);
  if (valid && lane == 0) d->bc[row] = s;
}

template <typename T, int FMT>
__global__ void __launch_bounds__(kVThreads) k_prolong(const LDesc<T>* __restrict__ descs) {
  MGD_PDL_TRIGGER();
  const LDesc<T>* d = descs + blockIdx.y;
  constexpr int TPR = FmtTraits<FMT>::tpr;
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  int row = g / TPR, lane = g % TPR;
  int n = d->n;
  if (((g & ~31LL) / TPR) >= n) return;
  bool valid = row < n;
  RowPre<T, kPre> R;
  row_load<T, FMT, kPre>(R, row, lane, valid, d->prp, d->pci, d->pv, nullptr, nullptr, nullptr);
  MGD_PDL_WAIT();
  MGD_SKIP_INACTIVE(d);
  XPlain<T> xf{d->xc};
  T s = row_finish<T, FMT, kPre>(R, valid, d->pci, d->pv, nullptr, nullptr, xf);
  if (valid && lane == 0) d->xt[row] += s;
}

// Multi-row forms of RESTRICT and PROLONG (FMT_CSR1X2, FMT_CSR1X4): one thread
// per row as in FMT_CSR1, each thread on the same lane of K adjacent 32-row
// groups.  A transfer row has few entries (one for a C point of P), so one row
// per thread leaves a warp one or two dependent loads in flight; here every
// gather of the K rows is issued before any sum is stored.  Each row sum takes
// its entries in CSR order, as in FMT_CSR1.
template <int K>
struct MrPre {
  static constexpr int pre = K >= 4 ? 2 : 3;  // entries per row loaded before the wait
};

template <typename T, int K, class XF>
__device__ __forceinline__ void mr_sums(const RowPre<T, MrPre<K>::pre> (&R)[K], int w, int lane, int n,
                                        const int* __restrict__ ci, const T* __restrict__ v, const XF& xf,
                                        T (&s)[K]) {
  constexpr int PRE = MrPre<K>::pre;
#pragma unroll
  for (int q = 0; q < K; ++q) {
    s[q] = T(0);
    if ((w * K + q) * 32 + lane < n) {
      const int first = R[q].p - PRE;
#pragma unroll
      for (int k = 0; k < PRE; ++k)
        if (first + k < R[q].e) s[q] += R[q].a[k] * xf(R[q].c[k]);
    }
  }
#pragma unroll
  for (int q = 0; q < K; ++q)
    if ((w * K + q) * 32 + lane < n)
      for (int p = R[q].p; p < R[q].e; ++p) s[q] += __ldg(v + p) * xf(__ldg(ci + p));
}

template <typename T, int K>
__global__ void __launch_bounds__(kVThreads) k_restrict_mr(const LDesc<T>* __restrict__ descs) {
  MGD_PDL_TRIGGER();
  const LDesc<T>* d = descs + blockIdx.y;
  constexpr int PRE = MrPre<K>::pre;
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  int w = g >> 5, lane = g & 31;
  int n = d->nc;
  if (w * 32 * K >= n) return;  // the whole warp is past the last row
  RowPre<T, PRE> R[K];
#pragma unroll
  for (int q = 0; q < K; ++q) {
    int r = (w * K + q) * 32 + lane;
    row_load<T, FMT_CSR1, PRE>(R[q], r, 0, r < n, d->rrp, d->rci, d->rv, nullptr, nullptr, nullptr);
  }
  MGD_PDL_WAIT();
  MGD_SKIP_INACTIVE(d);
  T s[K];
  mr_sums<T, K>(R, w, lane, n, d->rci, d->rv, XPlain<T>{d->r}, s);
#pragma unroll
  for (int q = 0; q < K; ++q) {
    int r = (w * K + q) * 32 + lane;
    if (r < n) d->bc[r] = s[q];
  }
}

template <typename T, int K>
__global__ void __launch_bounds__(kVThreads) k_prolong_mr(const LDesc<T>* __restrict__ descs) {
  MGD_PDL_TRIGGER();
  const LDesc<T>* d = descs + blockIdx.y;
  constexpr int PRE = MrPre<K>::pre;
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  int w = g >> 5, lane = g & 31;
  int n = d->n;
  if (w * 32 * K >= n) return;
  RowPre<T, PRE> R[K];
#pragma unroll
  for (int q = 0; q < K; ++q) {
    int r = (w * K + q) * 32 + lane;
    row_load<T, FMT_CSR1, PRE>(R[q], r, 0, r < n, d->prp, d->pci, d->pv, nullptr, nullptr, nullptr);
  }
  MGD_PDL_WAIT();
  MGD_SKIP_INACTIVE(d);
  T* xt = d->xt;
  T xo[K];
#pragma unroll
  for (int q = 0; q < K; ++q) {
    int r = (w * K + q) * 32 + lane;
    xo[q] = r < n ? xt[r] : T(0);
  }
  T s[K];
  mr_sums<T, K>(R, w, lane, n, d->pci, d->pv, XPlain<T>{d->xc}, s);
#pragma unroll
  for (int q = 0; q < K; ++q) {
    int r = (w * K + q) * 32 + lane;
    if (r < n) xt[r] = xo[q] + s[q];
  }
}

// stalled coarsest level, first l1-Jacobi sweep from zero: xt = D^-1 b
template <typename T>
__global__ void k_jac1(const LDesc<T>* __restrict__ descs) {
  MGD_PDL_ENTRY();
  const LDesc<T>* d = descs + blockIdx.y;
  MGD_SKIP_INACTIVE(d);
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < d->n) d->xt[i] = d->dinv[i] * d->b[i];
}

// coarsest level: x = A_L^{-1} b with the dense FP64 inverse (one CTA per subsystem)
template <typename T>
__global__ void k_coarse(const LDesc<T>* __restrict__ descs) {
  MGD_PDL_ENTRY();
  const LDesc<T>* d = descs + blockIdx.y;
  MGD_SKIP_INACTIVE(d);
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
    auto g_ = [&](int tpr) { return dim3(cdiv((long long)(maxrows) * tpr + 32, kVThreads), (ny)); }; \
    switch (fmt) {                                                                             \
      case FMT_SELL: launch_k(K<T, FMT_SELL>, dim3(g_(1)), dim3(kVThreads), 0, s, descs); break;                  \
      case FMT_CSR1: launch_k(K<T, FMT_CSR1>, dim3(g_(1)), dim3(kVThreads), 0, s, descs); break;                  \
      case FMT_CSR2: launch_k(K<T, FMT_CSR2>, dim3(g_(2)), dim3(kVThreads), 0, s, descs); break;                  \
      case FMT_CSR4: launch_k(K<T, FMT_CSR4>, dim3(g_(4)), dim3(kVThreads), 0, s, descs); break;                  \
      case FMT_CSR8: launch_k(K<T, FMT_CSR8>, dim3(g_(8)), dim3(kVThreads), 0, s, descs); break;                  \
      case FMT_CSR16: launch_k(K<T, FMT_CSR16>, dim3(g_(16)), dim3(kVThreads), 0, s, descs); break;               \
      default: launch_k(K<T, FMT_CSR32>, dim3(g_(32)), dim3(kVThreads), 0, s, descs); break;                      \
    }                                                                                          \
  } while (0)

template <typename T>
void launch_phase(int phase, int fmtA, int fmtRP, const LDesc<T>* d_descs, int ndesc, int maxrows, cudaStream_t s) {
  if (ndesc <= 0 || maxrows <= 0) return;
  int rp = fmtRP == FMT_SELL ? FMT_CSR1 : fmtRP;
  switch (phase) {
    case PH_PRE:
      if (fmtA == FMT_SELL2)
        launch_k(k_pre_sk<T, 2>, dim3(cdiv((long long)cdiv(maxrows, 64) * 32, kVThreads), ndesc), dim3(kVThreads), 0,
                 s, d_descs);
      else if (fmtA == FMT_SELL4)
        launch_k(k_pre_sk<T, 4>, dim3(cdiv((long long)cdiv(maxrows, 128) * 32, kVThreads), ndesc), dim3(kVThreads), 0,
                 s, d_descs);
      else
        MGD_DISPATCH_FMT(k_pre, fmtA, maxrows, ndesc, s, d_descs);
      break;
    case PH_POST:
      if (fmtA == FMT_SELL2)
        launch_k(k_post_sk<T, 2>, dim3(cdiv((long long)cdiv(maxrows, 64) * 32, kVThreads), ndesc), dim3(kVThreads), 0,
                 s, d_descs);
      else if (fmtA == FMT_SELL4)
        launch_k(k_post_sk<T, 4>, dim3(cdiv((long long)cdiv(maxrows, 128) * 32, kVThreads), ndesc), dim3(kVThreads), 0,
                 s, d_descs);
      else
        MGD_DISPATCH_FMT(k_post, fmtA, maxrows, ndesc, s, d_descs);
      break;
    case PH_RESTRICT:
      if (rp == FMT_CSR1X2)
        launch_k(k_restrict_mr<T, 2>, dim3(cdiv((long long)cdiv(maxrows, 64) * 32, kVThreads), ndesc),
                 dim3(kVThreads), 0, s, d_descs);
      else if (rp == FMT_CSR1X4)
        launch_k(k_restrict_mr<T, 4>, dim3(cdiv((long long)cdiv(maxrows, 128) * 32, kVThreads), ndesc),
                 dim3(kVThreads), 0, s, d_descs);
      else
        MGD_DISPATCH_FMT(k_restrict, rp, maxrows, ndesc, s, d_descs);
      break;
    case PH_PROLONG:
      if (rp == FMT_CSR1X2)
        launch_k(k_prolong_mr<T, 2>, dim3(cdiv((long long)cdiv(maxrows, 64) * 32, kVThreads), ndesc),
                 dim3(kVThreads), 0, s, d_descs);
      else if (rp == FMT_CSR1X4)
        launch_k(k_prolong_mr<T, 4>, dim3(cdiv((long long)cdiv(maxrows, 128) * 32, kVThreads), ndesc),
                 dim3(kVThreads), 0, s, d_descs);
      else
        MGD_DISPATCH_FMT(k_prolong, rp, maxrows, ndesc, s, d_descs);
      break;
    case PH_JAC1: launch_k(k_jac1<T>, dim3(dim3(cdiv(maxrows, kVThreads), ndesc)), dim3(kVThreads), 0, s, d_descs); break;
    case PH_COARSE:
      // one 1024-thread CTA per subsystem: a warp per row of the dense inverse
      launch_k(k_coarse<T>, dim3(dim3(1, ndesc)), dim3(1024), sizeof(double) * maxrows, s, d_descs);
      break;
  }
  MGD_LAUNCH_CHECK();
}

template void launch_phase<double>(int, int, int, const LDesc<double>*, int, int, cudaStream_t);
template void launch_phase<float>(int, int, int, const LDesc<float>*, int, int, cudaStream_t);

// ---------------------------------------------------------------- Gauss-Seidel smoothing (Section 3.1)
// Multicolour Gauss-Seidel in C/F order.  Down: the first sweep from a zero
// iterate (xt = b / a_ii on sweep 0's points, 0 elsewhere), then sweeps
// 1 .. nk-1, then r = b - A xt.  Up (after the prolongation): sweeps
// nk-1 .. 0.  A sweep updates its points in place: they are uncoupled, so
// every point reads only values of other sweeps.  x is the same buffer as xt
// on these levels.
template <typename T>
__global__ void k_gs_first(const LDesc<T>* __restrict__ descs) {
  MGD_PDL_ENTRY();
  const LDesc<T>* d = descs + blockIdx.y;
  MGD_SKIP_INACTIVE(d);
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < d->n) d->xt[i] = d->key[i] == 0 ? d->b[i] * d->gdinv[i] : T(0);
}

// step t of the down (up == 0: sweep t) or up (up == 1: sweep nk-1-t)
// smoothing.  FMT_SELL reads the level's sweep-ordered SELL copy (coalesced
// rows; position q of the sweep is row perm[q]); the CSR formats read A's
// rows through perm with TPR threads per row.
template <typename T, int FMT>
__global__ void __launch_bounds__(kVThreads) k_gs_sweep(const LDesc<T>* __restrict__ descs, int t, int up) {
  MGD_PDL_ENTRY();
  const LDesc<T>* d = descs + blockIdx.y;
  MGD_SKIP_INACTIVE(d);
  if (FMT == FMT_SELL && d->gsptr == nullptr) return;  // no sweep-ordered copy (never planned so)
  constexpr int TPR = FmtTraits<FMT>::tpr;
  const int nk = d->nk;
  const int k = up ? nk - 1 - t : t;
  if (k < 0 || k >= nk) return;
  const int seg = d->koff[k], cnt = d->koff[k + 1] - seg;
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  int idx = g / TPR, lane = g % TPR;
  if (((g & ~31) / TPR) >= cnt) return;  // whole warp past the sweep's last point
  bool valid = idx < cnt;
  int q = seg + idx;
  int row = valid ? d->perm[q] : 0;
  XPlain<T> xf{d->xt};
  T s = FMT == FMT_SELL ? row_dot<T, FMT>(q, lane, valid, nullptr, nullptr, nullptr, d->gsptr, d->gsci, d->gsv, xf)
                        : row_dot<T, FMT>(row, lane, valid, d->rp, d->ci, d->v, nullptr, nullptr, nullptr, xf);
  if (valid && lane == 0) d->xt[row] = d->xt[row] + (d->b[row] - s) * d->gdinv[row];
}

// r = b - A xt after the down sweeps (the level's A layout)
template <typename T, int FMT>
__global__ void __launch_bounds__(kVThreads) k_gs_resid(const LDesc<T>* __restrict__ descs) {
  MGD_PDL_TRIGGER();
  const LDesc<T>* d = descs + blockIdx.y;
  constexpr int TPR = FmtTraits<FMT>::tpr;
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  int row = g / TPR, lane = g % TPR;
  int n = d->n;
  if (((g & ~31) / TPR) >= n) return;
  bool valid = row < n;
  RowPre<T, kPre> R;
  row_load<T, FMT, kPre>(R, row, lane, valid, d->rp, d->ci, d->v, d->sptr, d->sci, d->sv);
  MGD_PDL_WAIT();
  MGD_SKIP_INACTIVE(d);
  XPlain<T> xf{d->xt};
  T s = row_finish<T, FMT, kPre>(R, valid, d->ci, d->v, d->sci, d->sv, xf);
  if (valid && lane == 0) d->r[row] = d->b[row] - s;
}

template <typename T>
void launch_gs_first(const LDesc<T>* d, int nd, int maxrows, cudaStream_t s) {
  if (nd <= 0 || maxrows <= 0) return;
  launch_k(k_gs_first<T>, dim3(cdiv(maxrows, kVThreads), nd), dim3(kVThreads), 0, s, d);
  MGD_LAUNCH_CHECK();
}

template <typename T>
void launch_gs_sweep(int fmt, const LDesc<T>* d, int nd, int maxrows, int t, int up, cudaStream_t s) {
  if (nd <= 0 || maxrows <= 0) return;
  auto g = [&](int tpr) { return dim3(cdiv((long long)maxrows * tpr + 32, kVThreads), nd); };
  switch (fmt) {
    case FMT_SELL: launch_k(k_gs_sweep<T, FMT_SELL>, g(1), dim3(kVThreads), 0, s, d, t, up); break;
    case FMT_CSR1: launch_k(k_gs_sweep<T, FMT_CSR1>, g(1), dim3(kVThreads), 0, s, d, t, up); break;
    case FMT_CSR2: launch_k(k_gs_sweep<T, FMT_CSR2>, g(2), dim3(kVThreads), 0, s, d, t, up); break;
    case FMT_CSR4: launch_k(k_gs_sweep<T, FMT_CSR4>, g(4), dim3(kVThreads), 0, s, d, t, up); break;
    default: launch_k(k_gs_sweep<T, FMT_CSR8>, g(8), dim3(kVThreads), 0, s, d, t, up); break;
  }
  MGD_LAUNCH_CHECK();
}

template <typename T>
void launch_gs_resid(int fmtA, const LDesc<T>* d, int nd, int maxrows, cudaStream_t s) {
  if (nd <= 0 || maxrows <= 0) return;
  if (fmtA == FMT_SELL2 || fmtA == FMT_SELL4) fmtA = FMT_SELL;  // multi-slice forms: l1-Jacobi phases only
  MGD_DISPATCH_FMT(k_gs_resid, fmtA, maxrows, nd, s, d);
  MGD_LAUNCH_CHECK();
}

template void launch_gs_first<double>(const LDesc<double>*, int, int, cudaStream_t);
template void launch_gs_first<float>(const LDesc<float>*, int, int, cudaStream_t);
template void launch_gs_sweep<double>(int, const LDesc<double>*, int, int, int, int, cudaStream_t);
template void launch_gs_sweep<float>(int, const LDesc<float>*, int, int, int, int, cudaStream_t);
template void launch_gs_resid<double>(int, const LDesc<double>*, int, int, cudaStream_t);
template void launch_gs_resid<float>(int, const LDesc<float>*, int, int, cudaStream_t);

// ---------------------------------------------------------------- fused coarse levels
// All levels from the first fused level down to the coarsest, and back up,
// in one launch: one thread-block cluster per subsystem, the phases separated
// by the cluster's hardware barrier (release / acquire at cluster scope).
// Vectors written inside the kernel are read through L2 (__ldcg); matrices,
// which are read-only here, through the read-only path.  Rows are handled by
// groups of 4 lanes; every warp runs the same number of row steps so that the
// shuffles and barriers are reached by all threads.
namespace cg = cooperative_groups;

constexpr int kTailTpr = 4;

template <typename T, bool MUT>
__device__ __forceinline__ T tail_load(const T* p) {
  if (MUT) return __ldcg(p);
  return __ldg(p);
}

// sum_p a_ip x_{ci_p} over one CSR row, by a group of kTailTpr lanes
template <typename T>
__device__ __forceinline__ T tail_row(const int* __restrict__ rp, const int* __restrict__ ci, const T* __restrict__ v,
                                      const T* x, int row, int lane, bool valid) {
  T s = T(0);
  if (valid) {
    int b = __ldg(rp + row), e = __ldg(rp + row + 1);
    for (int p = b + lane; p < e; p += kTailTpr) s += __ldg(v + p) * __ldcg(x + __ldg(ci + p));
  }
#pragma unroll
  for (int o = kTailTpr / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

template <typename T>
__global__ void __launch_bounds__(kTailThreads) k_vtail(const TailSub<T>* __restrict__ subs) {
  MGD_PDL_ENTRY();
  cg::cluster_group cl = cg::this_cluster();
  const int cs = (int)cl.num_blocks();
  const TailSub<T> S = subs[blockIdx.x / cs];
  MGD_SKIP_INACTIVE(S.lev);  // the same flag for every CTA of the cluster
  const int rank = (int)cl.block_rank();
  const int lane = threadIdx.x % kTailTpr;
  const int gwarp = rank * (kTailThreads / 32) + (int)(threadIdx.x >> 5);
  const int nwarps = cs * (kTailThreads / 32);
  constexpr int kRowsPerWarp = 32 / kTailTpr;
  const int wrow = (threadIdx.x & 31) / kTailTpr;
  // rows r = step * nwarps * 8 + gwarp * 8 + wrow, the same step count for every warp
  auto for_rows = [&](int nrows, auto&& body) {
    int steps = (nrows + nwarps * kRowsPerWarp - 1) / (nwarps * kRowsPerWarp);
    for (int st = 0; st < steps; ++st) {
      int r = (st * nwarps + gwarp) * kRowsPerWarp + wrow;
      body(r, r < nrows);
    }
  };
  // one Gauss-Seidel sweep (index sw) of level d, in place on xt
  auto gs_sweep = [&](const LDesc<T>* d, int sw) {
    const int seg = __ldg(d->koff + sw), cnt = __ldg(d->koff + sw + 1) - seg;
    for_rows(cnt, [&](int r, bool ok) {
      int row = ok ? __ldg(d->perm + seg + r) : 0;
      T s = tail_row<T>(d->rp, d->ci, d->v, d->xt, row, lane, ok);
      if (ok && lane == 0) d->xt[row] = __ldcg(d->xt + row) + (__ldcg(d->b + row) - s) * __ldg(d->gdinv + row);
    });
  };
  const int L = S.nlev;
  for (int k = 0; k < L - 1; ++k) {
    const LDesc<T>* d = S.lev + k;
    const int n = d->n, nc = d->nc;
    const int nk = d->nk;
    if (nk > 0) {
      // Gauss-Seidel down: sweep 0 from zero, sweeps 1 .. nk-1, then r = b - A xt
      for_rows(n, [&](int r, bool ok) {
        if (ok && lane == 0)
          d->xt[r] = __ldg(d->key + r) == 0 ? __ldcg(d->b + r) * __ldg(d->gdinv + r) : T(0);
      });
      cl.sync();
      for (int sw = 1; sw < nk; ++sw) {
        gs_sweep(d, sw);
        cl.sync();
      }
      for_rows(n, [&](int r, bool ok) {
        T s = tail_row<T>(d->rp, d->ci, d->v, d->xt, r, lane, ok);
        if (ok && lane == 0) d->r[r] = __ldcg(d->b + r) - s;
      });
    } else {
      // pre-smoothing from zero + residual: xt = D^-1 b, r = b - (A D^-1) b
      for_rows(n, [&](int r, bool ok) {
        T s = tail_row<T>(d->rp, d->ci, d->vpre, d->b, r, lane, ok);
        if (ok && lane == 0) {
          T bi = __ldcg(d->b + r);
          d->xt[r] = __ldg(d->dinv + r) * bi;
          d->r[r] = bi - s;
        }
      });
    }
    cl.sync();
    for_rows(nc, [&](int r, bool ok) {  // restriction
      T s = tail_row<T>(d->rrp, d->rci, d->rv, d->r, r, lane, ok);
      if (ok && lane == 0) d->bc[r] = s;
    });
    cl.sync();
  }
  {
    const LDesc<T>* d = S.lev + (L - 1);
    if (S.coarse_lu) {  // x = A_L^{-1} b, one warp per row
      const int n = d->cn;
      for (int i = gwarp; i < n; i += nwarps) {
        const double* row = d->cinv + (size_t)i * n;
        double s = 0.0;
        for (int j = threadIdx.x & 31; j < n; j += 32) s += __ldg(row + j) * (double)__ldcg(d->b + j);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) d->x[i] = (T)s;
      }
    } else {  // two l1-Jacobi sweeps from zero
      const int n = d->n;
      for (int i = rank * kTailThreads + threadIdx.x; i < n; i += cs * kTailThreads)
        d->xt[i] = __ldg(d->dinv + i) * __ldcg(d->b + i);
      cl.sync();
      for_rows(n, [&](int r, bool ok) {
        T s = tail_row<T>(d->rp, d->ci, d->v, d->xt, r, lane, ok);
        if (ok && lane == 0) d->x[r] = __ldcg(d->xt + r) + __ldg(d->dinv + r) * (__ldcg(d->b + r) - s);
      });
    }
  }
  cl.sync();
  for (int k = L - 2; k >= 0; --k) {
    const LDesc<T>* d = S.lev + k;
    const int n = d->n;
    for_rows(n, [&](int r, bool ok) {  // prolongation
      T s = tail_row<T>(d->prp, d->pci, d->pv, d->xc, r, lane, ok);
      if (ok && lane == 0) d->xt[r] = __ldcg(d->xt + r) + s;
    });
    cl.sync();
    if (d->nk > 0) {  // Gauss-Seidel up: the opposite traversal, in place (x is xt)
      for (int sw = d->nk - 1; sw >= 0; --sw) {
        gs_sweep(d, sw);
        cl.sync();
      }
      continue;
    }
    for_rows(n, [&](int r, bool ok) {  // post-smoothing
      T s = tail_row<T>(d->rp, d->ci, d->v, d->xt, r, lane, ok);
      if (ok && lane == 0) d->x[r] = __ldcg(d->xt + r) + __ldg(d->dinv + r) * (__ldcg(d->b + r) - s);
    });
    cl.sync();
  }
}

template <typename T>
void launch_vtail(const TailSub<T>* d_subs, int nsub, int cs, cudaStream_t s) {
  if (nsub <= 0) return;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nsub * cs, 1, 1);
  cfg.blockDim = dim3(kTailThreads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  MGD_CUDA(cudaLaunchKernelEx(&cfg, k_vtail<T>, d_subs));
  MGD_LAUNCH_CHECK();
}

// whether a cluster of cs CTAs of the fused kernel fits the device (sizes
// above 8 are non-portable and are enabled on the kernel first)
template <typename T>
bool vtail_cluster_fits(int cs) {
  if (cs > 8 && cudaFuncSetAttribute(k_vtail<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs, 1, 1);
  cfg.blockDim = dim3(kTailThreads, 1, 1);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_vtail<T>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return n > 0;
}
template bool vtail_cluster_fits<double>(int);
template bool vtail_cluster_fits<float>(int);

template void launch_vtail<double>(const TailSub<double>*, int, int, cudaStream_t);
template void launch_vtail<float>(const TailSub<float>*, int, int, cudaStream_t);

}  // namespace mgd
