// setup_kernels.cu -- device kernels of the AMG setup phase and of the block
// extraction (Sections 3.1, 3.3-3.6).
//
// This translation unit is compiled with -fmad=false and writes every
// floating-point step with an explicit round-to-nearest intrinsic, so each
// product and sum is rounded once, in the order the method's definitions
// state.  The C/F splittings and coarse operators therefore do not depend on
// the thread mapping: every output entry is produced by one thread in a fixed
// order.
#include "mgd_internal.cuh"

namespace mgd {

// ------------------------------------------------------------------ scan
// per block of kThreads * 4 outputs: exclusive sums of in[0..n_in) followed
// by zeros (n outputs), and the block's total in bsum
template <typename IN, typename I>
__global__ void k_scan_block_i(const IN* in, int n_in, I* out, I* bsum, int n) {
  __shared__ I sh[kThreads];
  int base = blockIdx.x * kThreads * 4;
  I v[4];
  I tsum = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    int i = base + threadIdx.x * 4 + k;
    v[k] = i < n_in ? (I)in[i] : (I)0;
    tsum += v[k];
  }
  sh[threadIdx.x] = tsum;
  __syncthreads();
  for (int off = 1; off < kThreads; off <<= 1) {
    I t = threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  I run = sh[threadIdx.x] - tsum;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    int i = base + threadIdx.x * 4 + k;
    if (i < n) out[i] = run;
    run += v[k];
  }
  if (threadIdx.x == kThreads - 1) bsum[blockIdx.x] = sh[kThreads - 1];
}

template <typename I>
__global__ void k_scan_add(I* out, const I* boff, int n, I* total_out, const I* btotal) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += boff[i / (kThreads * 4)];
  if (i == 0 && total_out) *total_out = *btotal;
}

// one block: exclusive sums of in[0..n_in) followed by zeros, n outputs,
// in chunks of kOneThreads * 4 with a running carry
constexpr int kOneThreads = 1024;
constexpr int kOneMax = 8 * kOneThreads;  // sizes served by the single-block scan
template <typename IN, typename I>
__global__ void __launch_bounds__(kOneThreads) k_scan_one(const IN* in, int n_in, I* out, int n) {
  __shared__ I sh[kOneThreads];
  I carry = 0;
  for (int base = 0; base < n; base += kOneThreads * 4) {
    I v[4];
    I tsum = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      int i = base + threadIdx.x * 4 + k;
      v[k] = i < n_in ? (I)in[i] : (I)0;
      tsum += v[k];
    }
    sh[threadIdx.x] = tsum;
    __syncthreads();
    for (int off = 1; off < kOneThreads; off <<= 1) {
      I t = threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
      __syncthreads();
      sh[threadIdx.x] += t;
      __syncthreads();
    }
    I run = carry + sh[threadIdx.x] - tsum;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      int i = base + threadIdx.x * 4 + k;
      if (i < n) out[i] = run;
      run += v[k];
    }
    carry += sh[kOneThreads - 1];
    __syncthreads();
  }
}

// out[0..n_out): exclusive sums of in[0..n_in) followed by zeros: blocks of
// kThreads * 4, their totals scanned by one block (or again by this, for
// more than kOneMax blocks), then added back; the input is read in place
template <typename IN, typename I>
static void scan_big(const IN* in, int n_in, I* out, int n_out, cudaStream_t s, Scratch& sc) {
  const int nb = cdiv(n_out, kThreads * 4);
  I* bsum = sc.alloc<I>(nb);
  I* boff = sc.alloc<I>(nb);
  k_scan_block_i<IN, I><<<nb, kThreads, 0, s>>>(in, n_in, out, bsum, n_out);
  MGD_LAUNCH_CHECK();
  if (nb <= kOneMax) {
    k_scan_one<I, I><<<1, kOneThreads, 0, s>>>(bsum, nb, boff, nb);
    MGD_LAUNCH_CHECK();
  } else {
    scan_big<I, I>(bsum, nb, boff, nb, s, sc);
  }
  k_scan_add<I><<<cdiv(n_out, kThreads), kThreads, 0, s>>>(out, boff, n_out, nullptr, nullptr);
  MGD_LAUNCH_CHECK();
}

// out[0..n]: exclusive prefix sums of in[0..n), out[n] = total
void exclusive_scan(const int* in, int* out, int n, cudaStream_t s) {
  if (n + 1 <= kOneMax) {
    k_scan_one<int, int><<<1, kOneThreads, 0, s>>>(in, n, out, n + 1);
    MGD_LAUNCH_CHECK();
    return;
  }
  Scratch sc(s);
  scan_big<int, int>(in, n, out, n + 1, s, sc);
}

void launch_offsets64(const int* cnt, long long* off, int n, cudaStream_t s) {
  if (n + 1 <= kOneMax) {
    k_scan_one<int, long long><<<1, kOneThreads, 0, s>>>(cnt, n, off, n + 1);
    MGD_LAUNCH_CHECK();
    return;
  }
  Scratch sc(s);
  scan_big<int, long long>(cnt, n, off, n + 1, s, sc);
}

int read_int(const int* d, cudaStream_t s) {
  int h = 0;
  MGD_CUDA(cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s));
  MGD_CUDA(cudaStreamSynchronize(s));
  return h;
}

// ------------------------------------------------------------------ validation and block extraction
// flags: 0 column out of range / unsorted / duplicated, 1 off-block entry
// outside its cell, 2 missing or non-positive diagonal, 3 row pointer not a
// non-decreasing map onto [0, nnz] (the row's entries are then not read),
// 4 a value that is not finite
__global__ void k_validate(int n, int nnz, int N, int nc, const int* rp, const int* ci, const double* v, int* flags) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (i == 0 && rp[0] != 0) atomicOr(&flags[3], 1);
  if (i == n - 1 && rp[n] != nnz) atomicOr(&flags[3], 1);
  const int rb = rp[i], re = rp[i + 1];
  if (rb < 0 || re < rb || re > nnz) {
    atomicOr(&flags[3], 1);
    return;
  }
  int a = i / N, k = i - a * N;
  int prev = -1;
  bool diag = false;
  for (int p = rb; p < re; ++p) {
    int j = ci[p];
    if (j < 0 || j >= n || j <= prev) atomicOr(&flags[0], 1);
    prev = j;
    int b = j / N;
    if (b != a && j - b * N != k) atomicOr(&flags[1], 1);
    if (!isfinite(v[p])) atomicOr(&flags[4], 1);
    if (j == i) {
      diag = true;
      if (!(v[p] > 0.0)) atomicOr(&flags[2], 1);
    }
  }
  if (!diag) atomicOr(&flags[2], 1);
}

void launch_validate(int n, int nnz, int N, int nc, const int* rp, const int* ci, const double* v, int* flags,
                     cudaStream_t s) {
  k_validate<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, nnz, N, nc, rp, ci, v, flags);
  MGD_LAUNCH_CHECK();
}

// cnt[a*N+k]: same-block entries of row (a,k); pairs[a*nc+b] = 1 where D_ab exists
__global__ void k_block_count(int n, int N, int nc, const int* rp, const int* ci, int* cnt, int* pairs) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int a = i / N;
  int c = 0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    int b = ci[p] / N;
    if (b == a) ++c;
    else pairs[a * nc + b] = 1;
  }
  cnt[i] = c;
}

void launch_block_count(int n, int N, int nc, const int* rp, const int* ci, int* cnt, int* pairs, cudaStream_t s) {
  k_block_count<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, N, nc, rp, ci, cnt, pairs);
  MGD_LAUNCH_CHECK();
}

// brp: block-stacked row pointer over all n rows (block a's rows are a*N..a*N+N-1);
// block-local columns; couplings scattered into dtab[a*nc+b][k]
__global__ void k_block_fill(int n, int N, int nc, const int* rp, const int* ci, const double* v, const int* brp,
                             int* bci, double* bv, double** dtab) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int a = i / N, k = i - a * N;
  int q = brp[i];
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    int j = ci[p];
    int b = j / N;
    if (b == a) {
      bci[q] = j - a * N;
      bv[q] = v[p];
      ++q;
    } else {
      double* d = dtab[a * nc + b];
      if (d) d[k] = v[p];
    }
  }
}

void launch_block_fill(int n, int N, int nc, const int* rp, const int* ci, const double* v, const int* brp,
                       int* bci, double* bv, double** dtab, cudaStream_t s) {
  k_block_fill<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, N, nc, rp, ci, v, brp, bci, bv, dtab);
  MGD_LAUNCH_CHECK();
}

// row pointers of every diagonal block from the block-major row pointer brp
// of the concatenated blocks: rp_a[k] = brp[a N + k] - brp[a N]
__global__ void k_block_rowptr(int N, int nc, const int* brp, int* const* rps) {
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (long long)nc * (N + 1)) return;
  int a = (int)(g / (N + 1)), k = (int)(g % (N + 1));
  rps[a][k] = brp[(long long)a * N + k] - brp[(long long)a * N];
}

void launch_block_rowptr(int N, int nc, const int* brp, int* const* rps, cudaStream_t s) {
  long long tot = (long long)nc * (N + 1);
  k_block_rowptr<<<cdiv(tot, kThreads), kThreads, 0, s>>>(N, nc, brp, rps);
  MGD_LAUNCH_CHECK();
}

// the block boundaries brp[a N], a = 0 .. nc
__global__ void k_block_bounds(int N, int nc, const int* brp, int* out) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a <= nc) out[a] = brp[(long long)a * N];
}

void launch_block_bounds(int N, int nc, const int* brp, int* out, cudaStream_t s) {
  k_block_bounds<<<cdiv(nc + 1, kThreads), kThreads, 0, s>>>(N, nc, brp, out);
  MGD_LAUNCH_CHECK();
}

__global__ void k_diag_extract(int n, const int* rp, const int* ci, const double* v, double* d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double r = 0.0;
  for (int p = rp[i]; p < rp[i + 1]; ++p)
    if (ci[p] == i) r = v[p];
  d[i] = r;
}

void launch_diag_extract(int n, const int* rp, const int* ci, const double* v, double* d, cudaStream_t s) {
  k_diag_extract<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, rp, ci, v, d);
  MGD_LAUNCH_CHECK();
}

// Section 3.5 diagonal Schur approximations: a_kk -= (x_k * y_k) / z_k
__global__ void k_diag_modify(int n, const int* rp, const int* ci, double* v, const double* x, const double* y,
                              const double* z) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int p = rp[i]; p < rp[i + 1]; ++p)
    if (ci[p] == i) {
      double t = __dmul_rn(x[i], y[i]);
      t = __ddiv_rn(t, z[i]);
      v[p] = __dsub_rn(v[p], t);
    }
}

void launch_diag_modify(int n, const int* rp, const int* ci, double* v, const double* x, const double* y,
                        const double* z, cudaStream_t s) {
  k_diag_modify<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, rp, ci, v, x, y, z);
  MGD_LAUNCH_CHECK();
}

// Definition 2: rows with sum_j a_kj < theta a_kk (row sum left to right)
__global__ void k_gamma_wd(int n, const int* rp, const int* ci, const double* v, double theta, int* count) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double rs = 0.0, akk = 0.0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    rs = __dadd_rn(rs, v[p]);
    if (ci[p] == i) akk = v[p];
  }
  if (rs < __dmul_rn(theta, akk)) atomicAdd(count, 1);
}

void launch_gamma_wd(int n, const int* rp, const int* ci, const double* v, double theta, int* count,
                     cudaStream_t s) {
  k_gamma_wd<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, rp, ci, v, theta, count);
  MGD_LAUNCH_CHECK();
}

// Definition 1: rows with -d_kk <= theta a_kk
__global__ void k_gamma_wc(int n, const double* d, const double* diag, double theta, int* count) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (-d[i] <= __dmul_rn(theta, diag[i])) atomicAdd(count, 1);
}

void launch_gamma_wc(int n, const double* d, const double* diag, double theta, int* count, cudaStream_t s) {
  k_gamma_wc<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, d, diag, theta, count);
  MGD_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ strength of connection (Section 3.1)
__global__ void k_strength(int n, const int* rp, const int* ci, const double* v, double theta, uint8_t* S) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double mx = 0.0;
  for (int p = rp[i]; p < rp[i + 1]; ++p)
    if (ci[p] != i && -v[p] > mx) mx = -v[p];
  double thr = __dmul_rn(theta, mx);
  for (int p = rp[i]; p < rp[i + 1]; ++p) S[p] = (uint8_t)(ci[p] != i && mx > 0.0 && -v[p] >= thr);
}

void launch_strength(int n, const int* rp, const int* ci, const double* v, double theta, uint8_t* S,
                     cudaStream_t s) {
  k_strength<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, rp, ci, v, theta, S);
  MGD_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ PMIS
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
// u(seed, stream, i): i-th output of a splitmix64 stream keyed by (seed, stream)
__device__ __forceinline__ double splitmix_uniform(uint64_t seed, uint64_t stream, uint64_t i) {
  const uint64_t G = 0x9E3779B97F4A7C15ULL;
  uint64_t key = mix64(mix64(seed + G) + stream * G);
  uint64_t z = mix64(key + (i + 1) * G);
  return __dmul_rn((double)(z >> 11), 1.0 / 9007199254740992.0);
}

__global__ void k_count_st(int n, const int* rp, const int* ci, const uint8_t* S, int* cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int p = rp[i]; p < rp[i + 1]; ++p)
    if (S[p]) atomicAdd(&cnt[ci[p]], 1);
}

void launch_count_st(int n, const int* rp, const int* ci, const uint8_t* S, int* cnt, cudaStream_t s) {
  k_count_st<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, rp, ci, S, cnt);
  MGD_LAUNCH_CHECK();
}

__global__ void k_fill_st(int n, const int* rp, const int* ci, const uint8_t* S, const int* strp, int* cursor,
                          int* stci) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int p = rp[i]; p < rp[i + 1]; ++p)
    if (S[p]) {
      int j = ci[p];
      int q = strp[j] + atomicAdd(&cursor[j], 1);
      stci[q] = i;
    }
}

void launch_fill_st(int n, const int* rp, const int* ci, const uint8_t* S, const int* strp, int* cursor,
                    int* stci, cudaStream_t s) {
  k_fill_st<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, rp, ci, S, strp, cursor, stci);
  MGD_LAUNCH_CHECK();
}

// weights w_i = |S^T_i| + u_i; isolated points and points nobody depends on are F
__global__ void k_pmis_init(int n, const int* rp, const uint8_t* S, const int* cnt, unsigned long long seed,
                            int level, double* w, signed char* CF) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double u = splitmix_uniform(seed, 1000ULL + (uint64_t)level, (uint64_t)i);
  double wi = __dadd_rn((double)cnt[i], u);
  w[i] = wi;
  int ns = 0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) ns += S[p];
  if (ns == 0 && cnt[i] == 0) CF[i] = -1;
  else if (wi < 1.0) CF[i] = -1;
  else CF[i] = 0;
}

void launch_pmis_init(int n, const int* rp, const uint8_t* S, const int* cnt, unsigned long long seed, int level,
                      double* w, signed char* CF, cudaStream_t s) {
  k_pmis_init<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, rp, S, cnt, seed, level, w, CF);
  MGD_LAUNCH_CHECK();
}

// ---------------------------------------------------------------- Gauss-Seidel order (Section 3.1 smoother)
// Jones-Plassmann colouring of the symmetrised graph of A (neighbours from A's
// and A^T's rows), weights u_i of the counter generator on stream 2000+level.
// Each round reads the colours of the previous round (col) and writes all of
// them to next, so points coloured in the same round never see each other.
__global__ void k_colour_init(int n, unsigned long long seed, int level, double* w, int* col) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  w[i] = splitmix_uniform(seed, 2000ULL + (uint64_t)level, (uint64_t)i);
  col[i] = -1;
}

__device__ __forceinline__ bool colour_beaten(const int* rp, const int* ci, int i, const int* col, const double* w) {
  double wi = w[i];
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    int j = ci[p];
    if (j == i || col[j] >= 0) continue;
    double wj = w[j];
    if (wj > wi || (wj == wi && j > i)) return true;
  }
  return false;
}

__device__ __forceinline__ bool colour_taken(const int* rp, const int* ci, const int* trp, const int* tci, int i,
                                             const int* col, int c) {
  for (int p = rp[i]; p < rp[i + 1]; ++p)
    if (ci[p] != i && col[ci[p]] == c) return true;
  for (int p = trp[i]; p < trp[i + 1]; ++p)
    if (tci[p] != i && col[tci[p]] == c) return true;
  return false;
}

__global__ void k_colour_round(int n, const int* rp, const int* ci, const int* trp, const int* tci, const double* w,
                               const int* col, int* next, int* left) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (col[i] >= 0) {
    next[i] = col[i];
    return;
  }
  if (colour_beaten(rp, ci, i, col, w) || colour_beaten(trp, tci, i, col, w)) {
    next[i] = -1;
    atomicAdd(left, 1);
    return;
  }
  // the smallest colour no coloured neighbour has: a bit mask for colours < 64
  unsigned long long used = 0ULL;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    int c = col[ci[p]];
    if (ci[p] != i && c >= 0 && c < 64) used |= 1ULL << c;
  }
  for (int p = trp[i]; p < trp[i + 1]; ++p) {
    int c = col[tci[p]];
    if (tci[p] != i && c >= 0 && c < 64) used |= 1ULL << c;
  }
  int c;
  if (~used) {
    c = __ffsll((long long)~used) - 1;
  } else {
    c = 64;
    while (colour_taken(rp, ci, trp, tci, i, col, c)) ++c;
  }
  next[i] = c;
}

// raw sweep class (C: colour, F: ncol + colour) counts and the largest colour
__global__ void k_colour_max(int n, const int* col, int* mx) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicMax(mx, col[i]);
}
__global__ void k_key_count(int n, const int* col, const signed char* CF, int ncol, int* cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(cnt + (CF[i] == 1 ? 0 : ncol) + col[i], 1);
}
__global__ void k_key_assign(int n, const int* col, const signed char* CF, int ncol, const int* map, int* key) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) key[i] = map[(CF[i] == 1 ? 0 : ncol) + col[i]];
}

// perm[koff[k] ..): the points of sweep k in increasing index order, one block per sweep
constexpr int kPermThreads = 1024;
__global__ void __launch_bounds__(kPermThreads) k_key_perm(int n, const int* __restrict__ key,
                                                           const int* __restrict__ koff, int* __restrict__ perm) {
  __shared__ int wsum[kPermThreads / 32];
  __shared__ int wpre[kPermThreads / 32];
  __shared__ int total;
  const int k = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int base = koff[k];
  for (int start = 0; start < n; start += kPermThreads) {
    int i = start + threadIdx.x;
    bool f = i < n && key[i] == k;
    unsigned bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
      int acc = 0;
      for (int w = 0; w < kPermThreads / 32; ++w) {
        wpre[w] = acc;
        acc += wsum[w];
      }
      total = acc;
    }
    __syncthreads();
    if (f) perm[base + wpre[warp] + __popc(bal & ((1u << lane) - 1u))] = i;
    base += total;
    __syncthreads();
  }
}

void launch_colour_init(int n, unsigned long long seed, int level, double* w, int* col, cudaStream_t s) {
  k_colour_init<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, seed, level, w, col);
  MGD_LAUNCH_CHECK();
}
void launch_colour_round(int n, const int* rp, const int* ci, const int* trp, const int* tci, const double* w,
                         const int* col, int* next, int* left, cudaStream_t s) {
  k_colour_round<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, rp, ci, trp, tci, w, col, next, left);
  MGD_LAUNCH_CHECK();
}
void launch_colour_max(int n, const int* col, int* mx, cudaStream_t s) {
  k_colour_max<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, col, mx);
  MGD_LAUNCH_CHECK();
}
void launch_key_count(int n, const int* col, const signed char* CF, int ncol, int* cnt, cudaStream_t s) {
  k_key_count<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, col, CF, ncol, cnt);
  MGD_LAUNCH_CHECK();
}
void launch_key_assign(int n, const int* col, const signed char* CF, int ncol, const int* map, int* key,
                       cudaStream_t s) {
  k_key_assign<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, col, CF, ncol, map, key);
  MGD_LAUNCH_CHECK();
}
void launch_key_perm(int n, int nk, const int* key, const int* koff, int* perm, cudaStream_t s) {
  if (nk <= 0) return;
  k_key_perm<<<nk, kPermThreads, 0, s>>>(n, key, koff, perm);
  MGD_LAUNCH_CHECK();
}

// aggressive coarsening: C indicator, and the final marks of the first pass's
// C points from the second pass (C stays C, anything else becomes F)
__global__ void k_cf_flag(int n, const signed char* CF, int* flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = CF[i] == 1 ? 1 : 0;
}
__global__ void k_cf_compose(int n, signed char* CF, const int* cidx, const signed char* CF2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && CF[i] == 1) CF[i] = CF2[cidx[i]] == 1 ? 1 : -1;
}
void launch_cf_flag(int n, const signed char* CF, int* flag, cudaStream_t s) {
  k_cf_flag<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, CF, flag);
  MGD_LAUNCH_CHECK();
}
void launch_cf_compose(int n, signed char* CF, const int* cidx, const signed char* CF2, cudaStream_t s) {
  k_cf_compose<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, CF, cidx, CF2);
  MGD_LAUNCH_CHECK();
}

// rows of A in sweep order (row q of the copy is row perm[q]; each row's
// entries keep their order, so a row sum over the copy is the same sum)
__global__ void k_perm_row_len(int n, const int* perm, const int* rp, int* len) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) len[q] = rp[perm[q] + 1] - rp[perm[q]];
}
__global__ void k_perm_rows_fill(int n, const int* perm, const int* rp, const int* ci, const double* v,
                                 const int* prp, int* pci, double* pv) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  int i = perm[q], b = rp[i], e = rp[i + 1], o = prp[q];
  for (int p = b; p < e; ++p) {
    pci[o + p - b] = ci[p];
    pv[o + p - b] = v[p];
  }
}
void launch_perm_row_len(int n, const int* perm, const int* rp, int* len, cudaStream_t s) {
  k_perm_row_len<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, perm, rp, len);
  MGD_LAUNCH_CHECK();
}
void launch_perm_rows_fill(int n, const int* perm, const int* rp, const int* ci, const double* v, const int* prp,
                           int* pci, double* pv, cudaStream_t s) {
  k_perm_rows_fill<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, perm, rp, ci, v, prp, pci, pv);
  MGD_LAUNCH_CHECK();
}

// PMIS weights are count + u with u in [0, 1): finite and not negative, so
// their bit patterns order as the values do and compare on the integer pipe
__device__ __forceinline__ bool beats(const double* w, int i, int j) {
  const long long wi = __double_as_longlong(w[i]), wj = __double_as_longlong(w[j]);
  return wi > wj || (wi == wj && i > j);
}

// round part 1: undecided local maxima over S_i and S^T_i become C (newc)
__global__ void k_pmis_select(int n, const int* rp, const int* ci, const uint8_t* S, const int* strp,
                              const int* stci, const double* w, const signed char* CF, uint8_t* newc,
                              int* undecided) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *undecided = 0;  // counted by k_pmis_fmark, the next launch on the stream
  if (i >= n) return;
  uint8_t res = 0;
  if (CF[i] == 0) {
    bool ismax = true;
    for (int p = rp[i]; p < rp[i + 1] && ismax; ++p)
      if (S[p] && CF[ci[p]] == 0 && !beats(w, i, ci[p])) ismax = false;
    for (int p = strp[i]; p < strp[i + 1] && ismax; ++p)
      if (CF[stci[p]] == 0 && !beats(w, i, stci[p])) ismax = false;
    res = ismax;
  }
  newc[i] = res;
}

// round part 2: the points selected in part 1 become C; undecided points that
// strongly depend on a C point (an old one, or one selected in part 1) become
// F.  A neighbour's CF may change during this launch only from 0 to 1 (when
// it was selected, which newc shows as well) or from 0 to -1 (when it was not),
// so the test CF == 1 || newc reads the same either way.
__global__ void k_pmis_fmark(int n, const int* rp, const int* ci, const uint8_t* S, const uint8_t* newc,
                             signed char* CF, int* undecided) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (newc[i]) {
    CF[i] = 1;
    return;
  }
  if (CF[i] != 0) return;
  for (int p = rp[i]; p < rp[i + 1]; ++p)
    if (S[p] && (CF[ci[p]] == 1 || newc[ci[p]])) {
      CF[i] = -1;
      return;
    }
  atomicAdd(undecided, 1);
}

void launch_pmis_round(int n, const int* rp, const int* ci, const uint8_t* S, const int* strp, const int* stci,
                       const double* w, signed char* CF, uint8_t* newc, int* undecided, cudaStream_t s) {
  int nb = cdiv(n, kThreads);
  k_pmis_select<<<nb, kThreads, 0, s>>>(n, rp, ci, S, strp, stci, w, CF, newc, undecided);
  MGD_LAUNCH_CHECK();
  k_pmis_fmark<<<nb, kThreads, 0, s>>>(n, rp, ci, S, newc, CF, undecided);
  MGD_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ classical modified interpolation
__global__ void k_interp_count(int n, const int* rp, const int* ci, const uint8_t* S, const signed char* CF,
                               int* cnt, int* isc) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  isc[i] = CF[i] == 1;
  int c = 0;
  if (CF[i] == 1) c = 1;
  else
    for (int p = rp[i]; p < rp[i + 1]; ++p)
      if (S[p] && CF[ci[p]] == 1) ++c;
  cnt[i] = c;
}

void launch_interp_count(int n, const int* rp, const int* ci, const uint8_t* S, const signed char* CF, int* cnt,
                         int* isc, cudaStream_t s) {
  k_interp_count<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, rp, ci, S, CF, cnt, isc);
  MGD_LAUNCH_CHECK();
}

// Comparisons of binary64 values with zero on the integer pipe (an FP64
// compare issues on the FP64 pipe, slow on this part), exact for every input
// including +-0, +-inf and NaN: x > 0 iff the sign is clear and the magnitude
// bits lie in (0, inf]; x < 0 iff the sign is set and likewise; x == 0 iff
// every bit but the sign is clear.
__device__ __forceinline__ bool pos_f64(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0 && b <= 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool neg_f64(double x) {
  const long long m = __double_as_longlong(x) & 0x7fffffffffffffffLL;
  return __double_as_longlong(x) < 0 && m > 0 && m <= 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool zero_f64(double x) { return (__double_as_longlong(x) << 1) == 0; }

__device__ __forceinline__ bool opp_sign(double akm, double akk) { return pos_f64(akk) ? neg_f64(akm) : pos_f64(akm); }

// One thread per row.  Numerators start from a_ij (j in C_i, row order); strong
// F neighbours k distribute a_ik abar_kj / sum_{m in C_i} abar_km, or are lumped
// into the diagonal with the weak neighbours when that sum is zero;
// w_ij = -num_j / (a_ii + sum_W a_in).

// ------------------------------------------------------------------ extended+i interpolation
// (De Sterck, Falgout, Nolting, Yang 2008): the interpolatory set of an F point
// adds, to its strong C neighbours, the strong C neighbours of its strong F
// neighbours.  Three kernels: an upper bound on each set, the deduplicated set
// in construction order (strong C neighbours of i in row order, then for each
// strong F neighbour k in row order its strong C neighbours in row order), and
// the weights with the same operation order as the definition states.

__global__ void k_exti_ub(int n, const int* rp, const int* ci, const uint8_t* S, const signed char* CF,
                          const int* scount, int* ub) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (CF[i] == 1) {
    ub[i] = 1;
    return;
  }
  int c = scount[i];
  for (int p = rp[i]; p < rp[i + 1]; ++p)
    if (S[p] && CF[ci[p]] == -1) c += scount[ci[p]];
  ub[i] = c;
}

// binary search of j in the sorted list L[0..len)
__device__ __forceinline__ int find_sorted(const int* L, int len, int j) {
  int lo = 0, hi = len;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (L[mid] < j) lo = mid + 1;
    else hi = mid;
  }
  return lo < len && L[lo] == j ? lo : -1;
}

// insert j into the sorted list L[0..t) unless present; returns the new length
__device__ __forceinline__ int insert_sorted(int* L, int t, int j) {
  int lo = 0, hi = t;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (L[mid] < j) lo = mid + 1;
    else hi = mid;
  }
  if (lo < t && L[lo] == j) return t;
  for (int q = t; q > lo; --q) L[q] = L[q - 1];
  L[lo] = j;
  return t + 1;
}

// interpolatory set of each F row, kept sorted by fine index (the coarse
// indices then come out in order: they grow with the fine ones)
__global__ void k_exti_list(int n, const int* rp, const int* ci, const uint8_t* S, const signed char* CF,
                            const long long* off, int* list, int* len) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (CF[i] == 1) {
    len[i] = 1;
    return;
  }
  int* L = list + off[i];
  int t = 0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    int j = ci[p];
    if (S[p] && CF[j] == 1) t = insert_sorted(L, t, j);
  }
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    int k = ci[p];
    if (!(S[p] && CF[k] == -1)) continue;
    for (int q = rp[k]; q < rp[k + 1]; ++q) {
      int m = ci[q];
      if (S[q] && CF[m] == 1) t = insert_sorted(L, t, m);
    }
  }
  len[i] = t;
}

// Extended+i values in three passes that keep every sum's operand order of
// the row-sequential definition (and so its bits).  Rows of A have sorted
// columns, so a_kl is found by binary search in row k.
__device__ __forceinline__ int find_col(const int* rp, const int* ci, int k, int l) {
  int b = rp[k];
  int q = find_sorted(ci + b, rp[k + 1] - b, l);
  return q < 0 ? -1 : b + q;
}

// row index of every entry
__global__ void k_row_of(int n, const int* rp, int* rowof) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int p = rp[i]; p < rp[i + 1]; ++p) rowof[p] = i;
}

// pass 1, one thread per entry (i, k) of A with i an F point and k a strong F
// neighbour: the distribution sum over row k of the opposite-sign entries at i
// or at an interpolatory point of i, in row-k order
__global__ void k_exti_denom(int nnz, const int* rowof, const int* rp, const int* ci, const double* v,
                             const uint8_t* S, const signed char* CF, const long long* off, const int* list,
                             const int* len, const double* dg, double* den) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nnz) return;
  int i = rowof[p], k = ci[p];
  if (CF[i] == 1 || k == i || !(S[p] && CF[k] == -1)) return;
  const int* L = list + off[i];
  int nl = len[i];
  double akk = dg[k];
  double denom = 0.0;
  for (int q = rp[k]; q < rp[k + 1]; ++q) {
    int l = ci[q];
    if ((l == i || find_sorted(L, nl, l) >= 0) && opp_sign(v[q], akk)) denom = __dadd_rn(denom, v[q]);
  }
  den[p] = denom;
}

// pass 2, one thread per F row: the lumped diagonal, in row order
__global__ void k_exti_diag(int n, const int* rp, const int* ci, const double* v, const uint8_t* S,
                            const signed char* CF, const long long* off, const int* list, const int* len,
                            const double* dg, const double* den, double* diagv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || CF[i] == 1 || len[i] == 0) return;
  const int* L = list + off[i];
  int nl = len[i];
  double diag = 0.0;
  for (int p = rp[i]; p < rp[i + 1]; ++p)
    if (ci[p] == i) diag = v[p];
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    int k = ci[p];
    if (k == i) continue;
    double aik = v[p];
    if (S[p] && CF[k] == 1) continue;
    if (S[p] && CF[k] == -1) {
      double denom = den[p];
      if (zero_f64(denom)) {
        diag = __dadd_rn(diag, aik);
      } else {
        int q = find_col(rp, ci, k, i);
        if (q >= 0 && opp_sign(v[q], dg[k])) diag = __dadd_rn(diag, __ddiv_rn(__dmul_rn(aik, v[q]), denom));
      }
    } else if (find_sorted(L, nl, k) < 0) {
      diag = __dadd_rn(diag, aik);
    }
  }
  diagv[i] = diag;
}

// pass 3, one thread per entry of P: the numerator of interpolatory point l of
// row i (its direct coefficient, then the distributed strong-F terms in row
// order), the weight -num / diag, and the coarse column
__global__ void k_exti_value(int nnzp, const int* prowof, const int* prp, const int* rp, const int* ci,
                             const double* v, const uint8_t* S, const signed char* CF, const int* cidx,
                             const long long* off, const int* list, const double* dg, const double* den,
                             const double* diagv, int* pci, double* pv) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnzp) return;
  int i = prowof[e];
  if (CF[i] == 1) {
    pci[e] = cidx[i];
    pv[e] = 1.0;
    return;
  }
  int l = list[off[i] + (e - prp[i])];
  double num = 0.0;
  int pd = find_col(rp, ci, i, l);
  if (pd >= 0) num = v[pd];
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    int k = ci[p];
    if (k == i || !(S[p] && CF[k] == -1)) continue;
    double denom = den[p];
    if (zero_f64(denom)) continue;
    int q = find_col(rp, ci, k, l);
    if (q >= 0 && opp_sign(v[q], dg[k])) num = __dadd_rn(num, __ddiv_rn(__dmul_rn(v[p], v[q]), denom));
  }
  double diag = diagv[i];
  pci[e] = cidx[l];
  pv[e] = !zero_f64(diag) ? __ddiv_rn(-num, diag) : 0.0;
}

// Classical modified interpolation values in passes that keep the operand
// order of the row-sequential definition (so its bits): the strong C
// neighbours of each F row are written in row order (sorted: CSR columns are
// sorted), then a denominator per strong-F entry of A, the lumped diagonal per
// row, the value of each entry of P, and last the fine-to-coarse column map.
__global__ void k_cl_set(int n, const int* rp, const int* ci, const uint8_t* S, const signed char* CF,
                         const int* cidx, const int* prp, int* pci, double* pv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int base = prp[i];
  if (CF[i] == 1) {
    pci[base] = cidx[i];
    pv[base] = 1.0;
    return;
  }
  int t = 0;
  for (int p = rp[i]; p < rp[i + 1]; ++p)
    if (S[p] && CF[ci[p]] == 1) pci[base + t++] = ci[p];  // fine index until the last pass
}

__global__ void k_cl_denom(int nnz, const int* rowof, const int* rp, const int* ci, const double* v, const uint8_t* S,
                           const signed char* CF, const int* prp, const int* pci, const double* dg, double* den) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nnz) return;
  int i = rowof[p], k = ci[p];
  if (CF[i] == 1 || k == i || !(S[p] && CF[k] == -1)) return;
  const int* L = pci + prp[i];
  int nl = prp[i + 1] - prp[i];
  double akk = dg[k];
  double denom = 0.0;
  for (int q = rp[k]; q < rp[k + 1]; ++q)
    if (find_sorted(L, nl, ci[q]) >= 0 && opp_sign(v[q], akk)) denom = __dadd_rn(denom, v[q]);
  den[p] = denom;
}

__global__ void k_cl_diag(int n, const int* rp, const int* ci, const double* v, const uint8_t* S,
                          const signed char* CF, const int* prp, const double* den, double* diagv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || CF[i] == 1 || prp[i + 1] == prp[i]) return;
  double diag = 0.0;
  for (int p = rp[i]; p < rp[i + 1]; ++p)
    if (ci[p] == i) diag = v[p];
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    int k = ci[p];
    if (k == i) continue;
    if (S[p] && CF[k] == 1) continue;
    if (S[p] && CF[k] == -1) {
      if (zero_f64(den[p])) diag = __dadd_rn(diag, v[p]);
    } else {
      diag = __dadd_rn(diag, v[p]);  // weak neighbours: lumped
    }
  }
  diagv[i] = diag;
}

__global__ void k_cl_value(int nnzp, const int* prowof, const int* rp, const int* ci, const double* v,
                           const uint8_t* S, const signed char* CF, const int* pci, const double* dg,
                           const double* den, const double* diagv, double* pv) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnzp) return;
  int i = prowof[e];
  if (CF[i] == 1) return;
  int m = pci[e];
  double num = 0.0;
  int pd = find_col(rp, ci, i, m);
  if (pd >= 0) num = v[pd];
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    int k = ci[p];
    if (k == i || !(S[p] && CF[k] == -1)) continue;
    double denom = den[p];
    if (zero_f64(denom)) continue;
    int q = find_col(rp, ci, k, m);
    if (q >= 0 && opp_sign(v[q], dg[k])) num = __dadd_rn(num, __ddiv_rn(__dmul_rn(v[p], v[q]), denom));
  }
  double diag = diagv[i];
  pv[e] = !zero_f64(diag) ? __ddiv_rn(-num, diag) : 0.0;
}

__global__ void k_cl_columns(int nnzp, const int* prowof, const signed char* CF, const int* cidx, int* pci) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < nnzp && CF[prowof[e]] != 1) pci[e] = cidx[pci[e]];
}

void launch_interp_fill(int n, int nnz, const int* rp, const int* ci, const double* v, const uint8_t* S,
                        const signed char* CF, const int* cidx, const int* prp, int nnzp, int* pci, double* pv,
                        const double* dg, int* work_i, double* work_d, cudaStream_t s) {
  // work_i: nnz + nnzp ints (row of each entry of A, of P); work_d: nnz + n doubles
  int* rowof = work_i;
  int* prowof = work_i + nnz;
  double* den = work_d;
  double* diagv = work_d + nnz;
  k_cl_set<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, rp, ci, S, CF, cidx, prp, pci, pv);
  MGD_LAUNCH_CHECK();
  k_row_of<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, rp, rowof);
  MGD_LAUNCH_CHECK();
  k_row_of<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, prp, prowof);
  MGD_LAUNCH_CHECK();
  if (nnz > 0) {
    k_cl_denom<<<cdiv(nnz, kThreads), kThreads, 0, s>>>(nnz, rowof, rp, ci, v, S, CF, prp, pci, dg, den);
    MGD_LAUNCH_CHECK();
  }
  k_cl_diag<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, rp, ci, v, S, CF, prp, den, diagv);
  MGD_LAUNCH_CHECK();
  if (nnzp > 0) {
    k_cl_value<<<cdiv(nnzp, kThreads), kThreads, 0, s>>>(nnzp, prowof, rp, ci, v, S, CF, pci, dg, den, diagv, pv);
    MGD_LAUNCH_CHECK();
    k_cl_columns<<<cdiv(nnzp, kThreads), kThreads, 0, s>>>(nnzp, prowof, CF, cidx, pci);
    MGD_LAUNCH_CHECK();
  }
}

void launch_exti_ub(int n, const int* rp, const int* ci, const uint8_t* S, const signed char* CF, const int* scount,
                    int* ub, cudaStream_t s) {
  k_exti_ub<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, rp, ci, S, CF, scount, ub);
  MGD_LAUNCH_CHECK();
}
void launch_exti_list(int n, const int* rp, const int* ci, const uint8_t* S, const signed char* CF,
                      const long long* off, int* list, int* len, cudaStream_t s) {
  k_exti_list<<<cdiv(n, 128), 128, 0, s>>>(n, rp, ci, S, CF, off, list, len);
  MGD_LAUNCH_CHECK();
}
void launch_exti_fill(int n, int nnz, const int* rp, const int* ci, const double* v, const uint8_t* S,
                      const signed char* CF, const int* cidx, const long long* off, const int* list, const int* len,
                      const int* prp, int nnzp, int* pci, double* pv, const double* dg, int* work_i,
                      double* work_d, cudaStream_t s) {
  // work_i: nnz + nnzp ints (row of each entry of A, of P); work_d: nnz + n doubles (denominators, diagonals)
  int* rowof = work_i;
  int* prowof = work_i + nnz;
  double* den = work_d;
  double* diagv = work_d + nnz;
  k_row_of<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, rp, rowof);
  MGD_LAUNCH_CHECK();
  k_row_of<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, prp, prowof);
  MGD_LAUNCH_CHECK();
  if (nnz > 0) {
    k_exti_denom<<<cdiv(nnz, kThreads), kThreads, 0, s>>>(nnz, rowof, rp, ci, v, S, CF, off, list, len, dg, den);
    MGD_LAUNCH_CHECK();
  }
  k_exti_diag<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, rp, ci, v, S, CF, off, list, len, dg, den, diagv);
  MGD_LAUNCH_CHECK();
  if (nnzp > 0) {
    k_exti_value<<<cdiv(nnzp, kThreads), kThreads, 0, s>>>(nnzp, prowof, prp, rp, ci, v, S, CF, cidx, off, list,
                                                           dg, den, diagv, pci, pv);
    MGD_LAUNCH_CHECK();
  }
}

// ------------------------------------------------------------------ transpose
__global__ void k_transpose_count(int nnz, const int* ci, int* cnt) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < nnz) atomicAdd(&cnt[ci[p]], 1);
}

void launch_transpose_count(int nnz, const int* ci, int* cnt, cudaStream_t s) {
  if (nnz == 0) return;
  k_transpose_count<<<cdiv(nnz, kThreads), kThreads, 0, s>>>(nnz, ci, cnt);
  MGD_LAUNCH_CHECK();
}

__global__ void k_transpose_fill(int n, const int* rp, const int* ci, const double* v, const int* trp,
                                 int* cursor, int* tci, double* tv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    int j = ci[p];
    int q = trp[j] + atomicAdd(&cursor[j], 1);
    tci[q] = i;
    tv[q] = v[p];
  }
}

void launch_transpose_fill(int n, const int* rp, const int* ci, const double* v, const int* trp, int* cursor,
                           int* tci, double* tv, cudaStream_t s) {
  k_transpose_fill<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, rp, ci, v, trp, cursor, tci, tv);
  MGD_LAUNCH_CHECK();
}

// insertion sort of each row by column (columns of a row are distinct)
__global__ void k_sort_rows(int n, const int* rp, int* ci, double* v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int b = rp[i], e = rp[i + 1];
  for (int a = b + 1; a < e; ++a) {
    int cc = ci[a];
    double vv = v[a];
    int q = a - 1;
    while (q >= b && ci[q] > cc) {
      ci[q + 1] = ci[q];
      v[q + 1] = v[q];
      --q;
    }
    ci[q + 1] = cc;
    v[q + 1] = vv;
  }
}

void launch_sort_rows(int n, const int* rp, int* ci, double* v, cudaStream_t s) {
  k_sort_rows<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, rp, ci, v);
  MGD_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ SpGEMM C = X Y (Galerkin products)
// For entry (i, j) the products x_ik y_kj are summed in the order of k along
// row i of X, the first product initialising the sum: products are expanded
// in that order, stably sorted by column, and each run is summed left to right.
__global__ void k_spgemm_ub(int n, const int* xrp, const int* xci, const int* yrp, int* ub) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = 0;
  for (int p = xrp[i]; p < xrp[i + 1]; ++p) {
    int k = xci[p];
    c += yrp[k + 1] - yrp[k];
  }
  ub[i] = c;
}

void launch_spgemm_ub(int n, const int* xrp, const int* xci, const int* yrp, int* ub, cudaStream_t s) {
  k_spgemm_ub<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, xrp, xci, yrp, ub);
  MGD_LAUNCH_CHECK();
}

// One thread per output row, for rows whose result has at most kThrSlots
// columns: the products are taken in expansion order (k along row i of X,
// then row k of Y) and each is either added to the entry of its column --
// __dadd_rn(sum so far, product) -- or inserted as a new entry of a sorted
// list in shared memory.  Each column's sum thus runs over its products left
// to right in expansion order, the first product initialising it: the result
// of the stable sort + run sums below.  Rows with more columns, or more than
// kThrMaxProducts products, are listed for the warp kernel.
constexpr int kThrSlots = 32;
constexpr int kThrRows = 128;
constexpr int kThrMaxProducts = 1024;
constexpr int kThrBatch = 8;  // entries of a row of Y loaded ahead of the merge

// SLOTS: the column-list capacity per row.  Shared memory (12 SLOTS bytes per
// thread) bounds the resident blocks, so a product whose rows are short runs
// with fewer slots and more warps per SM; a row that needs more columns is
// listed for the warp kernel, which gives the same sums.
template <int SLOTS>
__global__ void __launch_bounds__(kThrRows) k_spgemm_thread(int n, const int* xrp, const int* xci, const double* xv,
                                                            const int* yrp, const int* yci, const double* yv,
                                                            const long long* off, int* tc, double* tv, int* cnt,
                                                            int* wrows, int* nw) {
  __shared__ int s_c[SLOTS][kThrRows];
  __shared__ double s_v[SLOTS][kThrRows];
  const int t = threadIdx.x;
  const int i = blockIdx.x * kThrRows + t;
  if (i >= n) return;
  const long long b = off[i];
  const int L = (int)(off[i + 1] - b);
  bool over = L > kThrMaxProducts;
  int u = 0;  // columns so far, ascending in s_c[0 .. u)
  const int xe = over ? xrp[i] : xrp[i + 1];
  // the row of Y for the next entry of X is located one entry ahead, and the
  // entries of a row of Y are loaded kThrBatch at a time before they are
  // merged, so the global loads overlap instead of waiting one by one; the
  // products are still merged in expansion order
  int p = xrp[i];
  int nk = p < xe ? xci[p] : 0;
  int nyb = p < xe ? yrp[nk] : 0, nye = p < xe ? yrp[nk + 1] : 0;
  for (; p < xe && !over; ++p) {
    const double x = xv[p];
    const int yb = nyb, ye = nye;
    if (p + 1 < xe) {
      nk = xci[p + 1];
      nyb = yrp[nk];
      nye = yrp[nk + 1];
    }
    for (int q0 = yb; q0 < ye && !over; q0 += kThrBatch) {
      int bc[kThrBatch];
      double bv[kThrBatch];
#pragma unroll
      for (int j = 0; j < kThrBatch; ++j)
        if (q0 + j < ye) {
          bc[j] = yci[q0 + j];
          bv[j] = yv[q0 + j];
        }
#pragma unroll
      for (int j = 0; j < kThrBatch; ++j) {
      if (q0 + j >= ye || over) break;
      const int c = bc[j];
      const double pr = __dmul_rn(x, bv[j]);
      int lo = 0, hi = u;  // first entry with column >= c
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (s_c[mid][t] < c) lo = mid + 1;
        else hi = mid;
      }
      if (lo < u && s_c[lo][t] == c) {
        s_v[lo][t] = __dadd_rn(s_v[lo][t], pr);
        continue;
      }
      if (u == SLOTS) {
        over = true;
        break;
      }
      for (int m = u; m > lo; --m) {
        s_c[m][t] = s_c[m - 1][t];
        s_v[m][t] = s_v[m - 1][t];
      }
      s_c[lo][t] = c;
      s_v[lo][t] = pr;
      ++u;
      }
    }
  }
  if (over) {
    wrows[atomicAdd(nw, 1)] = i;
    return;
  }
  for (int m = 0; m < u; ++m) {
    tc[b + m] = s_c[m][t];
    tv[b + m] = s_v[m][t];
  }
  cnt[i] = u;
}

// One warp per listed output row, in shared memory for rows with at most
// kWarpProducts products: products are expanded in order (k along row i of X,
// then row k of Y), ranked by a stable counting sort on the column (ties keep
// their expansion order), and each run of equal columns is summed left to
// right by one lane.  Rows with up to kLongProducts products are listed for
// k_spgemm_long (a block per row); longer ones run the same three steps
// (expand, stable insertion sort, run sums) on one lane in global memory.
constexpr int kWarpProducts = 256;
constexpr int kSpgWarps = 4;
constexpr int kLongProducts = 8192;
constexpr int kLongThreads = 1024;

__device__ __forceinline__ void spgemm_warp_row(int i, int lane, const int* xrp, const int* xci, const double* xv,
                                                const int* yrp, const int* yci, const double* yv,
                                                const long long* off, int* tc, double* tv, int* cnt, int* longrows,
                                                int* nlong, int* col, double* val, int* scol, double* sval) {
  const long long b = off[i];
  const int L = (int)(off[i + 1] - b);
  if (L > kWarpProducts && L <= kLongProducts) {
    if (lane == 0) longrows[atomicAdd(nlong, 1)] = i;
    return;
  }
  if (L > kWarpProducts) {
    if (lane != 0) return;
    long long t = b;
    for (int p = xrp[i]; p < xrp[i + 1]; ++p) {
      int k = xci[p];
      double x = xv[p];
      for (int q = yrp[k]; q < yrp[k + 1]; ++q) {
        tc[t] = yci[q];
        tv[t] = __dmul_rn(x, yv[q]);
        ++t;
      }
    }
    long long e = t;
    for (long long a = b + 1; a < e; ++a) {
      int cc = tc[a];
      double vv = tv[a];
      long long q = a - 1;
      while (q >= b && tc[q] > cc) {
        tc[q + 1] = tc[q];
        tv[q + 1] = tv[q];
        --q;
      }
      tc[q + 1] = cc;
      tv[q + 1] = vv;
    }
    long long w = b;
    for (long long a = b; a < e;) {
      int cc = tc[a];
      double acc = tv[a];
      long long q = a + 1;
      while (q < e && tc[q] == cc) {
        acc = __dadd_rn(acc, tv[q]);
        ++q;
      }
      tc[w] = cc;
      tv[w] = acc;
      ++w;
      a = q;
    }
    cnt[i] = (int)(w - b);
    return;
  }
  // expansion: lane t takes entry t of a 32-entry chunk of row i of X; a warp
  // prefix sum of the Y row lengths places each lane's products, so the
  // expansion order (k along row i, then row k of Y) is unchanged
  int p0 = 0;
  const int xe = xrp[i + 1];
  for (int c = xrp[i]; c < xe; c += 32) {
    int p = c + lane;
    int yb = 0, len = 0;
    double x = 0.0;
    if (p < xe) {
      int k = xci[p];
      x = xv[p];
      yb = yrp[k];
      len = yrp[k + 1] - yb;
    }
    int incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    int at = p0 + incl - len;
    for (int q = 0; q < len; ++q) {
      col[at + q] = yci[yb + q];
      val[at + q] = __dmul_rn(x, yv[yb + q]);
    }
    p0 += __shfl_sync(0xffffffffu, incl, 31);
  }
  __syncwarp();
  for (int p = lane; p < L; p += 32) {  // stable rank by column
    int c = col[p], r = 0;
    for (int t = 0; t < L; ++t) {
      int ct = col[t];
      r += (ct < c) || (ct == c && t < p);
    }
    scol[r] = c;
    sval[r] = val[p];
  }
  __syncwarp();
  int base = 0;  // unique columns before this chunk
  for (int c0 = 0; c0 < L; c0 += 32) {
    int p = c0 + lane;
    bool start = p < L && (p == 0 || scol[p] != scol[p - 1]);
    unsigned m = __ballot_sync(0xffffffffu, start);
    if (start) {
      int u = base + __popc(m & ((1u << lane) - 1u));
      double acc = sval[p];
      int q = p + 1;
      while (q < L && scol[q] == scol[p]) {
        acc = __dadd_rn(acc, sval[q]);
        ++q;
      }
      tc[b + u] = scol[p];
      tv[b + u] = acc;
    }
    base += __popc(m);
  }
  if (lane == 0) cnt[i] = base;
}

__global__ void __launch_bounds__(32 * kSpgWarps) k_spgemm_warp(const int* xrp, const int* xci, const double* xv,
                                                                const int* yrp, const int* yci, const double* yv,
                                                                const long long* off, int* tc, double* tv, int* cnt,
                                                                const int* wrows, const int* nw, int* longrows,
                                                                int* nlong) {
  __shared__ int s_col[kSpgWarps][kWarpProducts];
  __shared__ double s_val[kSpgWarps][kWarpProducts];
  __shared__ int s_scol[kSpgWarps][kWarpProducts];
  __shared__ double s_sval[kSpgWarps][kWarpProducts];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nrows = *nw;
  for (int w = blockIdx.x * kSpgWarps + warp; w < nrows; w += gridDim.x * kSpgWarps)
    spgemm_warp_row(wrows[w], lane, xrp, xci, xv, yrp, yci, yv, off, tc, tv, cnt, longrows, nlong, s_col[warp],
                    s_val[warp], s_scol[warp], s_sval[warp]);
}


// One block per listed row (kWarpProducts < L <= kLongProducts): products
// expanded in order into shared memory with the key (column << 32 | position),
// a bitonic sort of the keys (the position makes it stable), then the runs of
// equal columns summed left to right, as in the warp kernel.
__global__ void __launch_bounds__(kLongThreads) k_spgemm_long(const int* xrp, const int* xci, const double* xv,
                                                              const int* yrp, const int* yci, const double* yv,
                                                              const long long* off, int* tc, double* tv, int* cnt,
                                                              const int* longrows, const int* nlong) {
  extern __shared__ unsigned long long sm_key[];  // kLongProducts keys, then kLongProducts values
  double* sm_val = reinterpret_cast<double*>(sm_key + kLongProducts);
  __shared__ int s_start[kLongThreads];
  __shared__ int s_flag[kLongThreads];
  const int tid = threadIdx.x;
  const int rows = *nlong;
  for (int r = blockIdx.x; r < rows; r += gridDim.x) {
    const int i = longrows[r];
    const long long b = off[i];
    const int L = (int)(off[i + 1] - b);
    const int x0 = xrp[i], nx = xrp[i + 1] - x0;
    // expansion offsets of the entries of row i of X (products of entry p start at s_start[p])
    for (int c0 = 0; c0 < nx; c0 += kLongThreads) {  // rows of X are short; chunked for safety
      __syncthreads();
      if (tid == 0) {
        int acc = c0 == 0 ? 0 : s_start[kLongThreads - 1] + (yrp[xci[x0 + c0 - 1] + 1] - yrp[xci[x0 + c0 - 1]]);
        for (int p = c0; p < nx && p < c0 + kLongThreads; ++p) {
          s_start[p - c0] = acc;
          int k = xci[x0 + p];
          acc += yrp[k + 1] - yrp[k];
        }
      }
      __syncthreads();
      for (int p = c0; p < nx && p < c0 + kLongThreads; ++p) {
        int k = xci[x0 + p];
        double x = xv[x0 + p];
        int yb = yrp[k], len = yrp[k + 1] - yb, t0 = s_start[p - c0];
        for (int q = tid; q < len; q += kLongThreads) {
          int t = t0 + q;
          sm_key[t] = ((unsigned long long)(unsigned)yci[yb + q] << 32) | (unsigned)t;
          sm_val[t] = __dmul_rn(x, yv[yb + q]);
        }
      }
    }
    int P2 = 1;
    while (P2 < L) P2 <<= 1;
    for (int t = L + tid; t < P2; t += kLongThreads) sm_key[t] = ~0ULL;
    __syncthreads();
    for (int k = 2; k <= P2; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int t = tid; t < P2; t += kLongThreads) {
          int u = t ^ j;
          if (u > t) {
            unsigned long long a = sm_key[t], c = sm_key[u];
            bool up = (t & k) == 0;
            if ((a > c) == up) {
              sm_key[t] = c;
              sm_key[u] = a;
            }
          }
        }
        __syncthreads();
      }
    // run heads, their ranks (chunked block scan), and the run sums
    int base = 0;
    for (int c0 = 0; c0 < L; c0 += kLongThreads) {
      int t = c0 + tid;
      int head = 0;
      if (t < L) head = t == 0 || (sm_key[t] >> 32) != (sm_key[t - 1] >> 32);
      s_flag[tid] = head;
      __syncthreads();
      for (int o = 1; o < kLongThreads; o <<= 1) {  // inclusive scan
        int v = tid >= o ? s_flag[tid - o] : 0;
        __syncthreads();
        s_flag[tid] += v;
        __syncthreads();
      }
      if (head) {
        int u = base + s_flag[tid] - 1;
        unsigned col = (unsigned)(sm_key[t] >> 32);
        double acc = sm_val[(unsigned)sm_key[t]];
        int q = t + 1;
        while (q < L && (unsigned)(sm_key[q] >> 32) == col) {
          acc = __dadd_rn(acc, sm_val[(unsigned)sm_key[q]]);
          ++q;
        }
        tc[b + u] = (int)col;
        tv[b + u] = acc;
      }
      base += s_flag[kLongThreads - 1];
      __syncthreads();
    }
    if (tid == 0) cnt[i] = base;
    __syncthreads();
  }
}

void launch_spgemm_expand(int n, const int* xrp, const int* xci, const double* xv, const int* yrp,
                          const int* yci, const double* yv, const long long* off, int* tc, double* tv, int* cnt,
                          int* work, cudaStream_t s, long long mean_products_hint) {
  // work: 2n + 2 ints (list of long rows, their count, list of the warp
  // kernel's rows, their count)
  int* nlong = work + n;
  int* wrows = work + n + 1;
  int* nw = work + 2 * n + 1;
  MGD_CUDA(cudaMemsetAsync(nlong, 0, sizeof(int), s));
  MGD_CUDA(cudaMemsetAsync(nw, 0, sizeof(int), s));
  if (n <= 0) return;
  // list size from the mean number of products per row (the upper bound of
  // its columns): the finest level's A P (about 17 products, at most ~19
  // columns on the 3-D workloads) takes 16 slots, its R (A P) 24
  const long long tot = mean_products_hint;
  if (tot > 0 && tot <= 24LL * n)
    k_spgemm_thread<16><<<cdiv(n, kThrRows), kThrRows, 0, s>>>(n, xrp, xci, xv, yrp, yci, yv, off, tc, tv, cnt, wrows,
                                                               nw);
  else if (tot > 0 && tot <= 96LL * n)
    k_spgemm_thread<24><<<cdiv(n, kThrRows), kThrRows, 0, s>>>(n, xrp, xci, xv, yrp, yci, yv, off, tc, tv, cnt, wrows,
                                                               nw);
  else
    k_spgemm_thread<kThrSlots><<<cdiv(n, kThrRows), kThrRows, 0, s>>>(n, xrp, xci, xv, yrp, yci, yv, off, tc, tv, cnt,
                                                                      wrows, nw);
  MGD_LAUNCH_CHECK();
  // the listed rows, a grid-stride loop over the list (its length stays on the device)
  k_spgemm_warp<<<152 * 8, 32 * kSpgWarps, 0, s>>>(xrp, xci, xv, yrp, yci, yv, off, tc, tv, cnt, wrows, nw, work,
                                                    nlong);
  MGD_LAUNCH_CHECK();
  static const size_t smem = (size_t)kLongProducts * (sizeof(unsigned long long) + sizeof(double));
  static const cudaError_t attr =
      cudaFuncSetAttribute(k_spgemm_long, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  MGD_CUDA(attr);
  k_spgemm_long<<<152, kLongThreads, smem, s>>>(xrp, xci, xv, yrp, yci, yv, off, tc, tv, cnt, work, nlong);
  MGD_LAUNCH_CHECK();
}

// copy each row's result to its final place: 8 lanes per row, consecutive
// lanes on consecutive entries
constexpr int kCompactLanes = 8;
__global__ void k_spgemm_compact(int n, const long long* off, const int* tc, const double* tv, const int* crp,
                                 int* cci, double* cv) {
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int i = (int)(g / kCompactLanes), lane = (int)(g % kCompactLanes);
  if (i >= n) return;
  long long b = off[i];
  int o = crp[i], len = crp[i + 1] - o;
  for (int k = lane; k < len; k += kCompactLanes) {
    cci[o + k] = tc[b + k];
    cv[o + k] = tv[b + k];
  }
}

void launch_spgemm_compact(int n, const long long* off, const int* tc, const double* tv, const int* crp, int* cci,
                           double* cv, cudaStream_t s) {
  k_spgemm_compact<<<cdiv((long long)n * kCompactLanes, kThreads), kThreads, 0, s>>>(n, off, tc, tv, crp, cci, cv);
  MGD_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ smoother diagonals, coarsest inverse
// dinv = 1 / sum_j |a_ij|; dinv32, when given, the same rounded to FP32
__global__ void k_l1_dinv(int n, const int* rp, const double* v, double* dinv, float* dinv32) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) s = __dadd_rn(s, fabs(v[p]));
  const double d = __ddiv_rn(1.0, s);
  dinv[i] = d;
  if (dinv32) dinv32[i] = (float)d;
}

void launch_l1_dinv(int n, const int* rp, const double* v, double* dinv, cudaStream_t s, float* dinv32) {
  k_l1_dinv<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, rp, v, dinv, dinv32);
  MGD_LAUNCH_CHECK();
}

__global__ void k_diag_inv(int n, const int* rp, const int* ci, const double* v, double* dinv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double d = 1.0;
  for (int p = rp[i]; p < rp[i + 1]; ++p)
    if (ci[p] == i) d = v[p];
  dinv[i] = __ddiv_rn(1.0, d);
}

void launch_diag_inv(int n, const int* rp, const int* ci, const double* v, double* dinv, cudaStream_t s) {
  k_diag_inv<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, rp, ci, v, dinv);
  MGD_LAUNCH_CHECK();
}

__global__ void k_densify(int n, const int* rp, const int* ci, const double* v, double* a) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int j = 0; j < n; ++j) a[(size_t)i * n + j] = 0.0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) a[(size_t)i * n + ci[p]] = v[p];
}

void launch_densify(int n, const int* rp, const int* ci, const double* v, double* a, cudaStream_t s) {
  k_densify<<<cdiv(n, 128), 128, 0, s>>>(n, rp, ci, v, a);
  MGD_LAUNCH_CHECK();
}

// Gaussian elimination with partial pivoting on one CTA (n <= a few hundred),
// then the explicit inverse column by column (one thread per unit vector).
__global__ void k_dense_inverse(int n, double* a, int* piv, double* inv, double* invT, int* status) {
  __shared__ int s_pr;
  __shared__ double s_best;
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      int pr = k;
      double best = fabs(a[(size_t)k * n + k]);
      for (int i = k + 1; i < n; ++i) {
        double t = fabs(a[(size_t)i * n + k]);
        if (t > best) {
          best = t;
          pr = i;
        }
      }
      s_pr = pr;
      s_best = best;
      piv[k] = pr;
    }
    __syncthreads();
    if (s_best == 0.0) {
      if (threadIdx.x == 0) *status = 1;
      return;
    }
    int pr = s_pr;
    if (pr != k)
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double t = a[(size_t)k * n + j];
        a[(size_t)k * n + j] = a[(size_t)pr * n + j];
        a[(size_t)pr * n + j] = t;
      }
    __syncthreads();
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) {
      double l = a[(size_t)i * n + k] / a[(size_t)k * n + k];
      a[(size_t)i * n + k] = l;
      for (int j = k + 1; j < n; ++j) a[(size_t)i * n + j] -= l * a[(size_t)k * n + j];
    }
    __syncthreads();
  }
  // column c of the inverse: solve A x = e_c
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    double* x = inv + (size_t)c * n;  // temporarily column-major in inv
    for (int i = 0; i < n; ++i) x[i] = (i == c) ? 1.0 : 0.0;
    for (int k = 0; k < n; ++k)
      if (piv[k] != k) {
        double t = x[k];
        x[k] = x[piv[k]];
        x[piv[k]] = t;
      }
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < i; ++j) x[i] -= a[(size_t)i * n + j] * x[j];
    for (int i = n - 1; i >= 0; --i) {
      for (int j = i + 1; j < n; ++j) x[i] -= a[(size_t)i * n + j] * x[j];
      x[i] /= a[(size_t)i * n + i];
    }
  }
  __syncthreads();
  // inv holds columns: invT[c*n + i] = (A^{-1})_{ic} is the row-major transpose
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) invT[e] = inv[e];
  __syncthreads();
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int i = e / n, c = e % n;
    inv[(size_t)i * n + c] = invT[(size_t)c * n + i];
  }
}

// Gauss-Jordan on [A | I] in shared memory, one 1024-thread block (n <= kGjMax).
// The rows below the pivot are updated exactly as the LU elimination above
// does (l = a_ik / a_kk, a_ij -= l a_kj, no fused multiply-add in this unit),
// so the pivot rows and the singularity decision are those of k_dense_inverse;
// rows above the pivot are eliminated too, and the reduced rows are finally
// divided by their pivots.
constexpr int kGjThreads = 1024;
constexpr int kGjMax = 112;  // 2 n^2 doubles + n multipliers fit the opt-in shared memory
__global__ void __launch_bounds__(kGjThreads) k_dense_inverse_gj(int n, const double* __restrict__ a0, int* piv,
                                                                 double* inv, double* invT, int* status) {
  extern __shared__ double gj[];
  double* A = gj;          // n x n, row-major
  double* X = gj + n * n;  // n x n, row-major, starts as I
  double* L = X + n * n;   // multipliers of the current step
  __shared__ int s_pr;
  __shared__ double s_best;
  const int t = threadIdx.x;
  for (int e = t; e < n * n; e += kGjThreads) {
    A[e] = a0[e];
    X[e] = (e / n == e % n) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (t < 32) {  // pivot: largest |a_ik|, i >= k, first index on ties (as the sequential search)
      double best = -1.0;
      int pr = n;
      for (int i = k + t; i < n; i += 32) {
        double v = fabs(A[i * n + k]);
        if (v > best) {
          best = v;
          pr = i;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        double ob = __shfl_xor_sync(0xffffffffu, best, o);
        int op = __shfl_xor_sync(0xffffffffu, pr, o);
        if (ob > best || (ob == best && op < pr)) {
          best = ob;
          pr = op;
        }
      }
      if (t == 0) {
        s_pr = pr;
        s_best = best;
        piv[k] = pr;
      }
    }
    __syncthreads();
    if (s_best == 0.0) {
      if (t == 0) *status = 1;
      return;
    }
    const int pr = s_pr;
    if (pr != k)
      for (int j = t; j < 2 * n; j += kGjThreads) {
        double* M = j < n ? A : X;
        int c = j < n ? j : j - n;
        double tmp = M[k * n + c];
        M[k * n + c] = M[pr * n + c];
        M[pr * n + c] = tmp;
      }
    __syncthreads();
    for (int i = t; i < n; i += kGjThreads) L[i] = i == k ? 0.0 : __ddiv_rn(A[i * n + k], A[k * n + k]);
    __syncthreads();
    // every row but k: columns k+1.. of A and all of X (32 x 32 threads: rows by
    // thread row, columns by lane)
    const int wa = n - k - 1, w = wa + n;
    const int ty = t >> 5, tx = t & 31;
    for (int i = ty; i < n; i += kGjThreads / 32) {
      if (i == k) continue;
      const double li = L[i];
      for (int j = tx; j < w; j += 32) {
        if (j < wa) {
          int c = k + 1 + j;
          A[i * n + c] = __dsub_rn(A[i * n + c], __dmul_rn(li, A[k * n + c]));
        } else {
          int c = j - wa;
          X[i * n + c] = __dsub_rn(X[i * n + c], __dmul_rn(li, X[k * n + c]));
        }
      }
    }
    __syncthreads();
  }
  for (int e = t; e < n * n; e += kGjThreads) {
    int i = e / n, c = e % n;
    double v = __ddiv_rn(X[e], A[i * n + i]);
    inv[e] = v;
    invT[c * n + i] = v;
  }
}

void launch_dense_inverse(int n, double* a, int* piv, double* inv, double* invT, int* status, cudaStream_t s) {
  if (n <= kGjMax) {
    size_t smem = (size_t)(2 * n * n + n) * sizeof(double);
    static const cudaError_t attr = cudaFuncSetAttribute(
        k_dense_inverse_gj, cudaFuncAttributeMaxDynamicSharedMemorySize,
        (int)((size_t)(2 * kGjMax * kGjMax + kGjMax) * sizeof(double)));
    MGD_CUDA(attr);
    k_dense_inverse_gj<<<1, kGjThreads, smem, s>>>(n, a, piv, inv, invT, status);
    MGD_LAUNCH_CHECK();
    return;
  }
  k_dense_inverse<<<1, 128, 0, s>>>(n, a, piv, inv, invT, status);
  MGD_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ PCTL coarse operator, Eq. 3.3
__global__ void k_pctl_ac_count(int N, int nc, const int* const* brp, const int* const* bci, int* cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  // union of the row patterns of all diagonal blocks: count distinct columns
  int c = 0;
  for (int a = 0; a < nc; ++a)
    for (int p = brp[a][i]; p < brp[a][i + 1]; ++p) {
      int j = bci[a][p];
      bool seen = false;
      for (int b = 0; b < a && !seen; ++b)
        for (int q = brp[b][i]; q < brp[b][i + 1]; ++q)
          if (bci[b][q] == j) {
            seen = true;
            break;
          }
      if (!seen) ++c;
    }
  cnt[i] = c;
}

void launch_pctl_ac_count(int N, int nc, const int* const* brp, const int* const* bci, int* cnt, cudaStream_t s) {
  k_pctl_ac_count<<<cdiv(N, 128), 128, 0, s>>>(N, nc, brp, bci, cnt);
  MGD_LAUNCH_CHECK();
}

// values in the order of Eq. 3.3: sum_g p_g(i) a^g_ij p_g(j) + a^E_ij + p_I(i) a^I_ij p_I(j)
// + [i == j] (sum_g d_Eg p_g + sum_g p_g d_gE + d_EI p_I + p_I d_IE)
__global__ void k_pctl_ac_fill(int N, int nc, int G, const int* const* brp, const int* const* bci,
                               const double* const* bv, const double* const* p, const double* const* dtab,
                               const int* acrp, int* acci, double* acv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int base = acrp[i], len = 0;
  for (int a = 0; a < nc; ++a)
    for (int q = brp[a][i]; q < brp[a][i + 1]; ++q) {
      int j = bci[a][q];
      bool seen = false;
      for (int s = 0; s < len; ++s)
        if (acci[base + s] == j) {
          seen = true;
          break;
        }
      if (!seen) {
        // insert sorted
        int s = len - 1;
        while (s >= 0 && acci[base + s] > j) {
          acci[base + s + 1] = acci[base + s];
          --s;
        }
        acci[base + s + 1] = j;
        ++len;
      }
    }
  int E = G, I = G + 1;
  for (int s = 0; s < len; ++s) {
    int j = acci[base + s];
    double acc = 0.0;
    for (int g = 0; g < G; ++g)
      for (int q = brp[g][i]; q < brp[g][i + 1]; ++q)
        if (bci[g][q] == j) acc = __dadd_rn(acc, __dmul_rn(__dmul_rn(p[g][i], bv[g][q]), p[g][j]));
    for (int q = brp[E][i]; q < brp[E][i + 1]; ++q)
      if (bci[E][q] == j) acc = __dadd_rn(acc, bv[E][q]);
    for (int q = brp[I][i]; q < brp[I][i + 1]; ++q)
      if (bci[I][q] == j) acc = __dadd_rn(acc, __dmul_rn(__dmul_rn(p[I][i], bv[I][q]), p[I][j]));
    if (j == i) {
      for (int g = 0; g < G; ++g)
        if (dtab[E * nc + g]) acc = __dadd_rn(acc, __dmul_rn(dtab[E * nc + g][i], p[g][i]));
      for (int g = 0; g < G; ++g)
        if (dtab[g * nc + E]) acc = __dadd_rn(acc, __dmul_rn(p[g][i], dtab[g * nc + E][i]));
      if (dtab[E * nc + I]) acc = __dadd_rn(acc, __dmul_rn(dtab[E * nc + I][i], p[I][i]));
      if (dtab[I * nc + E]) acc = __dadd_rn(acc, __dmul_rn(p[I][i], dtab[I * nc + E][i]));
    }
    acv[base + s] = acc;
  }
}

void launch_pctl_ac_fill(int N, int nc, int G, const int* const* brp, const int* const* bci,
                         const double* const* bv, const double* const* p, const double* const* dtab,
                         const int* acrp, int* acci, double* acv, cudaStream_t s) {
  k_pctl_ac_fill<<<cdiv(N, 128), 128, 0, s>>>(N, nc, G, brp, bci, bv, p, dtab, acrp, acci, acv);
  MGD_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ SELL-32 construction
__global__ void k_sell_widths(int n, const int* rp, int* w) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  int nsl = (n + 31) / 32;
  if (s >= nsl) return;
  int mx = 0;
  for (int r = s * 32; r < min(n, s * 32 + 32); ++r) mx = max(mx, rp[r + 1] - rp[r]);
  w[s] = mx * 32;
}

void launch_sell_widths(int n, const int* rp, int* w, cudaStream_t s) {
  int nsl = (n + 31) / 32;
  k_sell_widths<<<cdiv(nsl, kThreads), kThreads, 0, s>>>(n, rp, w);
  MGD_LAUNCH_CHECK();
}

// padding entries: value 0 at the row's own column (self[r] when given: the
// original index of a row of a row-permuted copy).  With d given, svpre gets
// the column-scaled values a_ij d_j (A D^-1, rounded once in FP64, then to T).
template <typename T>
__global__ void k_sell_fill(int n, const int* rp, const int* ci, const double* v, const double* d,
                            const int* sptr, int* sci, T* sv, T* svpre, const int* selfmap) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  int nsl = (n + 31) / 32;
  if (r >= nsl * 32) return;
  int s = r >> 5, lane = r & 31;
  int base = sptr[s];
  int width = (sptr[s + 1] - base) >> 5;
  int len = r < n ? rp[r + 1] - rp[r] : 0;
  int b = r < n ? rp[r] : 0;
  int self = r < n ? (selfmap ? selfmap[r] : r) : 0;
  for (int j = 0; j < width; ++j) {
    int idx = base + j * 32 + lane;
    if (j < len) {
      int c = ci[b + j];
      double a = v[b + j];
      sci[idx] = c;
      sv[idx] = (T)a;
      if (svpre) svpre[idx] = (T)__dmul_rn(a, d[c]);
    } else {
      sci[idx] = self;
      sv[idx] = T(0);
      if (svpre) svpre[idx] = T(0);
    }
  }
}

template <typename T>
static void sell_fill(int n, const int* rp, const int* ci, const double* v, const double* d, const int* sptr,
                      int* sci, T* sv, T* svpre, cudaStream_t s, const int* selfmap) {
  int nsl = (n + 31) / 32;
  k_sell_fill<T><<<cdiv(nsl * 32, kThreads), kThreads, 0, s>>>(n, rp, ci, v, d, sptr, sci, sv, d ? svpre : nullptr,
                                                               selfmap);
  MGD_LAUNCH_CHECK();
}

void launch_sell_fill(int n, const int* rp, const int* ci, const double* v, const double* d, const int* sptr,
                      int* sci, double* sv, double* svpre, cudaStream_t s, const int* selfmap) {
  sell_fill<double>(n, rp, ci, v, d, sptr, sci, sv, svpre, s, selfmap);
}

void launch_sell_fill(int n, const int* rp, const int* ci, const double* v, const double* d, const int* sptr,
                      int* sci, float* sv, float* svpre, cudaStream_t s, const int* selfmap) {
  sell_fill<float>(n, rp, ci, v, d, sptr, sci, sv, svpre, s, selfmap);
}

// ------------------------------------------------------------------ column scaling A D^-1
// out = A D^-1 values (the FP64 product, rounded to T); vout, when given, the
// values themselves rounded to T (the FP32 copy of a level, in the same pass)
template <typename T>
__global__ void k_colscale(long long nnz, const int* ci, const double* v, const double* d, T* vout, T* out) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nnz) return;
  double a = v[p];
  if (vout) vout[p] = (T)a;
  if (out) out[p] = (T)__dmul_rn(a, d[ci[p]]);
}

void launch_colscale(long long nnz, const int* ci, const double* v, const double* d, double* out, cudaStream_t s) {
  if (nnz <= 0) return;
  k_colscale<double><<<cdiv(nnz, kThreads), kThreads, 0, s>>>(nnz, ci, v, d, nullptr, out);
  MGD_LAUNCH_CHECK();
}

void launch_colscale_f32(long long nnz, const int* ci, const double* v, const double* d, float* vout, float* out,
                         cudaStream_t s) {
  if (nnz <= 0) return;
  k_colscale<float><<<cdiv(nnz, kThreads), kThreads, 0, s>>>(nnz, ci, v, d, vout, d ? out : nullptr);
  MGD_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ adjoint gradient
__global__ void k_grad_vals(int n, const int* rp, const int* ci, const double* x, const double* lam, double* g) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double l = lam[i];
  for (int p = rp[i]; p < rp[i + 1]; ++p) g[p] = -l * x[ci[p]];
}

void launch_grad_vals(int n, const int* rp, const int* ci, const double* x, const double* lam, double* g,
                      cudaStream_t s) {
  k_grad_vals<<<cdiv(n, kThreads), kThreads, 0, s>>>(n, rp, ci, x, lam, g);
  MGD_LAUNCH_CHECK();
}

}  // namespace mgd
