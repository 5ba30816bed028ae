// mgd_internal.cuh -- internal structures and kernel launchers of the
// sm_103a solver library (not part of the C ABI).
#pragma once
#include <functional>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

namespace mgd {

// ------------------------------------------------------------------ errors
struct Error {
  int code;
  std::string msg;
};

#define MGD_CUDA(call)                                                                      \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      throw ::mgd::Error{7, std::string(#call) + ": " + cudaGetErrorString(e_) + " at " +   \
                                __FILE__ + ":" + std::to_string(__LINE__)};                 \
  } while (0)

// every kernel launch of the library is followed by this check, which also
// counts the launch (see mgd_kernel_launches)
extern long long g_kernel_launches;
#define MGD_LAUNCH_CHECK()                                         \
  do {                                                             \
    __atomic_add_fetch(&::mgd::g_kernel_launches, 1, __ATOMIC_RELAXED); \
    MGD_CUDA(cudaGetLastError());                                  \
  } while (0)

constexpr int kThreads = 256;

// Programmatic dependent launch: solve kernels are launched with the
// programmatic-stream-serialisation attribute; each waits for its predecessor
// grid (griddepcontrol.wait) before touching memory and then lets its own
// successor start launching, so launch latency overlaps the previous kernel.
// Without the attribute both instructions are no-ops.
#define MGD_PDL_ENTRY()                                         \
  do {                                                          \
    asm volatile("griddepcontrol.wait;" ::: "memory");          \
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); \
  } while (0)
// Split form for kernels that read setup-time data (operators, descriptors)
// before the wait: they let their successor launch at entry, load what no
// predecessor in the solve writes, then wait before the first read of a
// vector (or of an inner-loop flag) that a predecessor wrote.
#define MGD_PDL_TRIGGER() asm volatile("griddepcontrol.launch_dependents;" ::: "memory")
#define MGD_PDL_WAIT() asm volatile("griddepcontrol.wait;" ::: "memory")

extern thread_local bool tl_pdl;

template <typename... KArgs, typename... Args>
inline void launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = tl_pdl ? 1 : 0;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
  if (e != cudaSuccess) throw Error{7, std::string("kernel launch: ") + cudaGetErrorString(e)};
}

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// ------------------------------------------------------------------ memory
// Device memory of a context comes from its own stream-ordered memory pool
// (cudaMemPool with a high release threshold, so freed blocks stay cached and
// no allocation or free synchronises the device).
struct Pool {
  cudaMemPool_t pool = nullptr;
  void create(int device) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    MGD_CUDA(cudaMemPoolCreate(&pool, &props));
    unsigned long long thr = ~0ULL;
    MGD_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
  }
  void destroy() {
    if (pool) cudaMemPoolDestroy(pool);
    pool = nullptr;
  }
};

// the pool and (in setup worker threads) the stream of the calling thread
extern thread_local cudaMemPool_t tl_pool;
extern thread_local cudaStream_t tl_stream;

inline void* pool_alloc(cudaMemPool_t pool, size_t bytes, cudaStream_t s) {
  if (!pool) pool = tl_pool;
  void* p = nullptr;
  cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, s) : cudaMallocAsync(&p, bytes, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error{8, "device allocation of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e)};
  }
  return p;
}

// Allocations owned by a context, freed together at destroy / re-setup.
// Arrays are carved, 256-byte aligned, from slabs of the context's pool (the
// first 4 MiB, each next one twice the last, up to 1 GiB; an array above 256
// MiB gets a block of its own), so a setup makes a few dozen pool allocations
// instead of thousands and the release frees as many.  A slab is allocated on
// the arena's own stream, which is otherwise idle, and synchronised there
// before any array in it is handed out, so every stream may use it; arrays
// are never freed one by one.  Safe to use from the setup worker threads:
// each zeroes on its own stream and synchronises it before the memory is used
// elsewhere.
struct Arena {
  std::vector<void*> ptrs;          // slabs and separate blocks
  cudaStream_t stream = nullptr;    // the context stream (release)
  cudaMemPool_t pool = nullptr;
  cudaStream_t astream = nullptr;   // slab allocations
  std::mutex mu;
  char* cur = nullptr;              // free part of the current slab
  size_t left = 0;
  size_t next_slab = kSlabMin;
  static constexpr size_t kSlabMin = (size_t)4 << 20, kSlabMax = (size_t)1 << 30;
  static constexpr size_t kAlign = 256;
  template <typename T>
  T* alloc(size_t n, bool zero = false, cudaStream_t zs = nullptr) {
    const size_t bytes = (n ? n : 1) * sizeof(T);
    const size_t need = (bytes + kAlign - 1) & ~(kAlign - 1);
    cudaStream_t st = zs ? zs : (tl_stream ? tl_stream : stream);
    void* p;
    {
      std::lock_guard<std::mutex> lk(mu);
      if (need > kSlabMax / 4) {
        p = block_locked(need);
      } else {
        if (need > left) {
          size_t sz = next_slab;
          while (sz < need) sz *= 2;
          cur = static_cast<char*>(block_locked(sz));
          left = sz;
          next_slab = std::min(sz * 2, kSlabMax);
        }
        p = cur;
        cur += need;
        left -= need;
      }
    }
    if (zero) MGD_CUDA(cudaMemsetAsync(p, 0, bytes, st));
    return (T*)p;
  }
  void* block_locked(size_t bytes) {
    if (!astream) MGD_CUDA(cudaStreamCreateWithFlags(&astream, cudaStreamNonBlocking));
    void* p = pool_alloc(pool, bytes, astream);
    const cudaError_t e = cudaStreamSynchronize(astream);
    if (e != cudaSuccess) {
      cudaFreeAsync(p, astream);
      throw Error{8, std::string("device allocation failed: ") + cudaGetErrorString(e)};
    }
    ptrs.push_back(p);
    return p;
  }
  void release() {
    std::lock_guard<std::mutex> lk(mu);
    if (stream) cudaStreamSynchronize(stream);
    for (void* p : ptrs) cudaFreeAsync(p, stream);
    if (stream) cudaStreamSynchronize(stream);
    ptrs.clear();
    cur = nullptr;
    left = 0;
    next_slab = kSlabMin;
  }
  ~Arena() {
    if (astream) cudaStreamDestroy(astream);
  }
};

// Scratch memory of one setup worker thread, for the work it issues on its
// own stream: chunks of the context's pool (64 MiB first, doubling), handed out
// as a stack of 256-byte aligned blocks.  A freed block is marked dead and the
// stack top rewinds over dead blocks, so memory comes back in the order the
// scopes close; a block reused this way is only ever touched by later work on
// the same stream, which the stream orders after the work that used it
// before.  This replaces one pool allocation and one pool free per scratch
// array, which the concurrent setup threads otherwise serialise on.
struct ScratchRegion {
  struct Chunk {
    char* base;
    size_t size;
  };
  struct Blk {
    int chunk;
    size_t off, bytes;
    bool live;
  };
  cudaStream_t stream = nullptr;
  cudaMemPool_t pool = nullptr;
  std::vector<Chunk> chunks;
  std::vector<Blk> stack;
  static constexpr size_t kChunkMin = (size_t)64 << 20;
  ScratchRegion(cudaStream_t s, cudaMemPool_t p) : stream(s), pool(p) {}
  void* alloc(size_t bytes) {
    const size_t need = (bytes + 255) & ~(size_t)255;
    int c = stack.empty() ? 0 : stack.back().chunk;
    size_t off = stack.empty() ? 0 : stack.back().off + stack.back().bytes;
    if (!chunks.empty() && off + need > chunks[c].size) {
      ++c;
      off = 0;
    }
    if (c >= (int)chunks.size() || chunks[c].size < need) {
      size_t sz = std::max(kChunkMin, chunks.empty() ? need : 2 * chunks.back().size);
      while (sz < need) sz *= 2;
      if (c < (int)chunks.size()) {  // too small for this block: replaced (stream-ordered free)
        cudaFreeAsync(chunks[c].base, stream);
        chunks[c] = Chunk{static_cast<char*>(pool_alloc(pool, sz, stream)), sz};
      } else {
        chunks.push_back(Chunk{static_cast<char*>(pool_alloc(pool, sz, stream)), sz});
      }
    }
    stack.push_back(Blk{c, off, need, true});
    return chunks[c].base + off;
  }
  void free(void* p) {
    for (size_t k = stack.size(); k-- > 0;)
      if (chunks[stack[k].chunk].base + stack[k].off == p && stack[k].live) {
        stack[k].live = false;
        break;
      }
    while (!stack.empty() && !stack.back().live) stack.pop_back();
  }
  ~ScratchRegion() {
    for (auto& ch : chunks) cudaFreeAsync(ch.base, stream);
  }
};

// the scratch region of the calling setup worker thread (nullptr elsewhere)
extern thread_local ScratchRegion* tl_region;

// Scratch allocations for one setup step (stream-ordered, freed at scope
// exit): from the calling worker's region when they are for its stream, else
// from the pool
struct Scratch {
  std::vector<void*> ptrs;
  cudaStream_t stream;
  cudaMemPool_t pool;
  ScratchRegion* region;
  explicit Scratch(cudaStream_t s, cudaMemPool_t p = nullptr)
      : stream(s), pool(p ? p : tl_pool), region(tl_region && tl_region->stream == s ? tl_region : nullptr) {}
  template <typename T>
  T* alloc(size_t n) {
    const size_t bytes = (n ? n : 1) * sizeof(T);
    void* p = region ? region->alloc(bytes) : pool_alloc(pool, bytes, stream);
    ptrs.push_back(p);
    return (T*)p;
  }
  ~Scratch() {
    for (size_t k = ptrs.size(); k-- > 0;) {
      if (region) region->free(ptrs[k]);
      else cudaFreeAsync(ptrs[k], stream);
    }
  }
};

// ------------------------------------------------------------------ matrices
struct Csr {  // device CSR, FP64 values
  int n = 0, m = 0, nnz = 0;
  int* rp = nullptr;
  int* ci = nullptr;
  double* v = nullptr;
};

// sparse-kernel formats chosen per level by the autotuner
enum Fmt { FMT_SELL = 0, FMT_CSR1 = 1, FMT_CSR2 = 2, FMT_CSR4 = 3, FMT_CSR8 = 4, FMT_CSR16 = 5, FMT_CSR32 = 6,
           FMT_SELL2 = 7, FMT_SELL4 = 8,     // SELL-32 with each thread on the same lane of 2 / 4 adjacent
                                             // slices (l1-Jacobi smoothing phases only)
           FMT_CSR1X2 = 9, FMT_CSR1X4 = 10 };  // CSR, one thread per row, each thread on the same lane of
                                               // 2 / 4 adjacent 32-row groups (restriction, prolongation only)

struct Sell {  // sliced ELL, slice height 32, column-major inside a slice
  int n = 0, nslices = 0;
  long long nstored = 0;
  int* sptr = nullptr;  // [nslices+1] element offsets (multiples of 32)
  int* ci = nullptr;
  double* v = nullptr;
  float* v32 = nullptr;
  double* vpre = nullptr;   // values scaled by the column's l1 inverse
  float* vpre32 = nullptr;
};

// Per-level device view used by the V-cycle kernels (T = double or float).
template <typename T>
struct LDesc {
  int n, nc;
  // operator (CSR and, when built, SELL)
  const int* rp;
  const int* ci;
  const T* v;
  const int* sptr;
  const int* sci;
  const T* sv;
  const T* dinv;
  // A D^-1 (columns scaled by the smoother diagonal): the pre-smoothing
  // residual b - A D^-1 b then costs one multiply-add per nonzero
  const T* vpre;
  const T* svpre;
  // prolongation P (n x nc) and restriction R = P^T (nc x n), CSR
  const int* prp;
  const int* pci;
  const T* pv;
  const int* rrp;
  const int* rci;
  const T* rv;
  // vectors
  T* b;   // right-hand side of this level
  T* x;   // output of this level's cycle
  T* xt;  // smoothed iterate before post-smoothing
  T* r;   // residual
  T* bc;  // next level's right-hand side
  T* xc;  // next level's output
  // coarsest level: dense inverse (FP64, row-major cn x cn)
  const double* cinv;
  int cn;
  // option #3 / multi-cycle loops: the subsystem's flag (nullptr: always
  // run); a V-cycle kernel skips a subsystem whose flag is 0
  const int* active;
  // Gauss-Seidel smoother (nk > 0): sweep index per row, the rows of sweep k
  // at perm[koff[k] .. koff[k+1]), and 1 / a_ii
  const int* key;
  const int* perm;
  const int* koff;
  int nk;
  const T* gdinv;
  // A's rows in sweep order as SELL-32 (row q = row perm[q], original columns)
  const int* gsptr;
  const int* gsci;
  const T* gsv;
};

// the V-cycle kernels' first statement after the dependency wait: leave a
// subsystem that its inner loop has already finished (uniform per CTA)
#define MGD_SKIP_INACTIVE(d) \
  do {                        \
    const int* a_ = (d)->active; \
    if (a_ && *a_ == 0) return; \
  } while (0)

// One subsystem's share of the fused coarse-level kernel: its level
// descriptors from the first fused level to its coarsest level.
template <typename T>
struct TailSub {
  const LDesc<T>* lev;  // device array, nlev entries (first = first fused level)
  int nlev;             // fused levels including the coarsest (>= 1)
  int coarse_lu;        // coarsest: 1 dense inverse, 0 two l1-Jacobi sweeps
};

// Block-level pointer reference: absolute, or relative to the current
// preconditioner input v / output z held in device memory (graph-safe).
struct PRef {
  int slot;          // 0: absolute, 1: v + off, 2: z + off
  long long off;
  double* abs;
};

struct IOSlots {
  const double* v;
  double* z;
};

constexpr int kMaxTerms = 32;
// a CONSUME and the PRODUCE after it fuse into one kernel when their
// descriptors fit its shared-memory tables
constexpr int kCpMaxCons = 64, kCpMaxProd = 64, kCpMaxTerms = 512;
template <typename T>
struct ProduceDesc {  // dst = (T)(a + sum_t s_t * d_t (.) w_t)
  T* dst;
  PRef a;             // a.slot == 0 && a.abs == nullptr: a = 0
  int nt;
  const double* d[kMaxTerms];  // nullptr: 1
  PRef w[kMaxTerms];
  double s[kMaxTerms];
};
template <typename T>
struct ConsumeDesc {  // dst = base + s * (double)x
  PRef dst;
  PRef base;          // null: 0
  double s;
  int unit;           // 1: s = +1, 2: s = -1 (applied without a multiply), 0: other
  const T* x;
};
template <typename T>
struct JacDesc {      // option #1: x = dinv (.) b
  T* x;
  const T* b;
  const T* dinv;
};

// One operator of a device-controlled inverse (Section 3.5): option #3
// (x = 0; x += V(rhs - A x) until ||rhs - A x|| <= tol ||rhs||, at most
// maxit cycles) or a fixed number of cycles (x = V rhs; x += V(rhs - A x)).
// The V-cycle reads b and writes x (the hierarchy's level-0 vectors).
template <typename T>
struct InnerDesc {
  const int* rp;   // level-0 operator, CSR
  const int* ci;
  const T* v;
  T* b;            // V-cycle input: the residual
  T* x;            // V-cycle output: the correction (the solution after the loop)
  T* rhs;          // the right-hand side, saved
  T* xacc;         // accumulated solution
  int n;
  int accurate;    // 1: option #3, 0: `count` cycles
  int count;
  int* active;     // read by the V-cycle kernels of this operator's hierarchy
};
// loop state of one INVERT step (device memory)
constexpr int kInnerParts = 608;  // partial-norm blocks per operator (4 per SM)
struct InnerCtl {
  int nops, maxit, guard;  // guard: hard cap on loop trips (>= every op's cap)
  double tol;
  double* part;            // nops x kInnerParts partial sums of squares
  double* nr0;             // ||rhs|| per op
  int* cycles;             // cycles of the current apply, per op
  long long* total;        // cycles since setup, per op
  int* trips;              // loop trips of the current apply
  int* any;                // 1 while some op is active (read by the host loop)
};

// ------------------------------------------------------------------ setup launchers (setup_kernels.cu)
void exclusive_scan(const int* in, int* out, int n, cudaStream_t s);  // out[0..n], out[n] = total
int read_int(const int* d, cudaStream_t s);
// FP64 multiply-add lane operations per second of the whole device (measured)
double measure_fp64_rate(cudaStream_t s);
long long check_conversions(cudaStream_t s);  // mismatches of the integer-pipe format conversions

void launch_validate(int n, int nnz, int N, int nc, const int* rp, const int* ci, const double* v, int* flags,
                     cudaStream_t s);
void launch_block_count(int n, int N, int nc, const int* rp, const int* ci, int* cnt, int* pairs, cudaStream_t s);
void launch_block_rowptr(int N, int nc, const int* brp, int* const* rps, cudaStream_t s);
void launch_block_bounds(int N, int nc, const int* brp, int* out, cudaStream_t s);
void launch_block_fill(int n, int N, int nc, const int* rp, const int* ci, const double* v, const int* brp,
                       int* bci, double* bv, double** dtab, cudaStream_t s);
void launch_diag_extract(int n, const int* rp, const int* ci, const double* v, double* d, cudaStream_t s);
void launch_diag_modify(int n, const int* rp, const int* ci, double* v, const double* x, const double* y,
                        const double* z, cudaStream_t s);
void launch_gamma_wd(int n, const int* rp, const int* ci, const double* v, double theta, int* count,
                     cudaStream_t s);
void launch_gamma_wc(int n, const double* d, const double* diag, double theta, int* count, cudaStream_t s);

void launch_strength(int n, const int* rp, const int* ci, const double* v, double theta, uint8_t* S,
                     cudaStream_t s);
void launch_count_st(int n, const int* rp, const int* ci, const uint8_t* S, int* cnt, cudaStream_t s);
void launch_fill_st(int n, const int* rp, const int* ci, const uint8_t* S, const int* strp, int* cursor,
                    int* stci, cudaStream_t s);
void launch_pmis_init(int n, const int* rp, const uint8_t* S, const int* cnt, unsigned long long seed, int level,
                      double* w, signed char* CF, cudaStream_t s);
void launch_pmis_round(int n, const int* rp, const int* ci, const uint8_t* S, const int* strp, const int* stci,
                       const double* w, signed char* CF, uint8_t* newc, int* undecided, cudaStream_t s);
void launch_colour_init(int n, unsigned long long seed, int level, double* w, int* col, cudaStream_t s);
void launch_colour_round(int n, const int* rp, const int* ci, const int* trp, const int* tci, const double* w,
                         const int* col, int* next, int* left, cudaStream_t s);
void launch_colour_max(int n, const int* col, int* mx, cudaStream_t s);
void launch_key_count(int n, const int* col, const signed char* CF, int ncol, int* cnt, cudaStream_t s);
void launch_key_assign(int n, const int* col, const signed char* CF, int ncol, const int* map, int* key,
                       cudaStream_t s);
void launch_key_perm(int n, int nk, const int* key, const int* koff, int* perm, cudaStream_t s);
void launch_cf_flag(int n, const signed char* CF, int* flag, cudaStream_t s);
void launch_cf_compose(int n, signed char* CF, const int* cidx, const signed char* CF2, cudaStream_t s);
void launch_perm_row_len(int n, const int* perm, const int* rp, int* len, cudaStream_t s);
void launch_perm_rows_fill(int n, const int* perm, const int* rp, const int* ci, const double* v, const int* prp,
                           int* pci, double* pv, cudaStream_t s);
void launch_interp_count(int n, const int* rp, const int* ci, const uint8_t* S, const signed char* CF, int* cnt,
                         int* isc, cudaStream_t s);
void launch_interp_fill(int n, int nnz, const int* rp, const int* ci, const double* v, const uint8_t* S,
                        const signed char* CF, const int* cidx, const int* prp, int nnzp, int* pci, double* pv,
                        const double* dg, int* work_i, double* work_d, cudaStream_t s);
void launch_exti_ub(int n, const int* rp, const int* ci, const uint8_t* S, const signed char* CF, const int* scount,
                    int* ub, cudaStream_t s);
void launch_exti_list(int n, const int* rp, const int* ci, const uint8_t* S, const signed char* CF,
                      const long long* off, int* list, int* len, cudaStream_t s);
void launch_exti_fill(int n, int nnz, const int* rp, const int* ci, const double* v, const uint8_t* S,
                      const signed char* CF, const int* cidx, const long long* off, const int* list, const int* len,
                      const int* prp, int nnzp, int* pci, double* pv, const double* dg, int* work_i,
                      double* work_d, cudaStream_t s);
void launch_transpose_count(int nnz, const int* ci, int* cnt, cudaStream_t s);
void launch_transpose_fill(int n, const int* rp, const int* ci, const double* v, const int* trp, int* cursor,
                           int* tci, double* tv, cudaStream_t s);
void launch_sort_rows(int n, const int* rp, int* ci, double* v, cudaStream_t s);
void launch_spgemm_ub(int n, const int* xrp, const int* xci, const int* yrp, int* ub, cudaStream_t s);
// total_products: the expansion's product count (sets the per-row list size)
void launch_spgemm_expand(int n, const int* xrp, const int* xci, const double* xv, const int* yrp,
                          const int* yci, const double* yv, const long long* off, int* tc, double* tv, int* cnt,
                          int* work, cudaStream_t s, long long total_products);  // work: 2n + 2 ints
void launch_spgemm_compact(int n, const long long* off, const int* tc, const double* tv, const int* crp,
                           int* cci, double* cv, cudaStream_t s);
void launch_l1_dinv(int n, const int* rp, const double* v, double* dinv, cudaStream_t s, float* dinv32 = nullptr);
void launch_diag_inv(int n, const int* rp, const int* ci, const double* v, double* dinv, cudaStream_t s);
void launch_densify(int n, const int* rp, const int* ci, const double* v, double* a, cudaStream_t s);
void launch_dense_inverse(int n, double* a, int* piv, double* inv, double* invT, int* status, cudaStream_t s);
void launch_pctl_ac_count(int N, int nc, const int* const* brp, const int* const* bci, int* cnt, cudaStream_t s);
void launch_pctl_ac_fill(int N, int nc, int G, const int* const* brp, const int* const* bci,
                         const double* const* bv, const double* const* p, const double* const* dtab,
                         const int* acrp, int* acci, double* acv, cudaStream_t s);
void launch_sell_widths(int n, const int* rp, int* w, cudaStream_t s);
// SELL-32 copy of a CSR matrix; with d given, svpre gets A D^-1 in the same pass
void launch_sell_fill(int n, const int* rp, const int* ci, const double* v, const double* d, const int* sptr,
                      int* sci, double* sv, double* svpre, cudaStream_t s, const int* selfmap = nullptr);
void launch_sell_fill(int n, const int* rp, const int* ci, const double* v, const double* d, const int* sptr,
                      int* sci, float* sv, float* svpre, cudaStream_t s, const int* selfmap = nullptr);
void launch_colscale(long long nnz, const int* ci, const double* v, const double* d, double* out, cudaStream_t s);
// FP32 values (vout) and FP32 A D^-1 (out, when d is given) of FP64 CSR values, one pass
void launch_colscale_f32(long long nnz, const int* ci, const double* v, const double* d, float* vout, float* out,
                         cudaStream_t s);
void launch_grad_vals(int n, const int* rp, const int* ci, const double* x, const double* lam, double* g,
                      cudaStream_t s);
void launch_offsets64(const int* cnt, long long* off, int n, cudaStream_t s);

// ------------------------------------------------------------------ solve launchers (solve_kernels.cu)
enum Phase { PH_PRE = 0, PH_RESTRICT = 1, PH_PROLONG = 2, PH_POST = 3, PH_COARSE = 4, PH_JAC1 = 5 };

template <typename T>
void launch_phase(int phase, int fmtA, int tprRP, const LDesc<T>* d_descs, int ndesc, int maxrows,
                  cudaStream_t s);
// Gauss-Seidel smoothing phases (levels with nk > 0)
template <typename T>
void launch_gs_first(const LDesc<T>* d, int nd, int maxrows, cudaStream_t s);
template <typename T>
void launch_gs_sweep(int fmt, const LDesc<T>* d, int nd, int maxrows, int t, int up, cudaStream_t s);
template <typename T>
void launch_gs_resid(int fmtA, const LDesc<T>* d, int nd, int maxrows, cudaStream_t s);
// fused coarse-level V-cycle: one thread-block cluster of `cs` CTAs per subsystem
template <typename T>
void launch_vtail(const TailSub<T>* d_subs, int nsub, int cs, cudaStream_t s);
constexpr int kTailThreads = 512;
template <typename T>
bool vtail_cluster_fits(int cs);

template <typename T>
void launch_produce(const ProduceDesc<T>* d, int nd, int N, const IOSlots* io, cudaStream_t s);
template <typename T>
void launch_consume(const ConsumeDesc<T>* d, int nd, int N, const IOSlots* io, cudaStream_t s);
template <typename T>
void launch_consume_produce(const ConsumeDesc<T>* cd, int ncd, const ProduceDesc<T>* pd, int npd, int N,
                            const IOSlots* io, cudaStream_t s);
template <typename T>
void launch_jacobi(const JacDesc<T>* d, int nd, int N, cudaStream_t s);
template <typename T>
void launch_residual(int fmt, int n, const int* rp, const int* ci, const T* v, const int* sptr, const int* sci,
                     const T* sv, const T* b, const T* x, T* r, cudaStream_t s);
template <typename T>
void launch_axpy(int n, T* y, const T* x, cudaStream_t s);  // y += x

// device-controlled inverse loop (one INVERT step, nd operators):
//   begin: rhs = b, xacc = 0, partial ||b||^2; ctl(first)
//   loop while any active: V-cycle; update (xacc += x); resid (b = rhs - A xacc,
//   partial ||b||^2); ctl
//   end: x = xacc, b = rhs, active = 1
// ctl sets the conditional node's value when use_cond (graph replay)
template <typename T>
void launch_inner_begin(const InnerDesc<T>* d, int nd, int maxn, const InnerCtl* ctl, cudaStream_t s);
template <typename T>
void launch_inner_update(const InnerDesc<T>* d, int nd, int maxn, cudaStream_t s);
template <typename T>
void launch_inner_resid(const InnerDesc<T>* d, int nd, int maxn, const InnerCtl* ctl, cudaStream_t s);
template <typename T>
void launch_inner_ctl(const InnerDesc<T>* d, int nd, const InnerCtl* ctl, int first, int use_cond,
                      cudaGraphConditionalHandle cond, cudaStream_t s);
template <typename T>
void launch_inner_end(const InnerDesc<T>* d, int nd, int maxn, cudaStream_t s);

void launch_spmv_f64(int fmt, int n, const int* rp, const int* ci, const double* v, const int* sptr,
                     const int* sci, const double* sv, const double* x, double* y, cudaStream_t s);
void launch_resid_f64(int fmt, int n, const int* rp, const int* ci, const double* v, const int* sptr,
                      const int* sci, const double* sv, const double* b, const double* x, double* r,
                      cudaStream_t s);
void launch_set_io(IOSlots* io, const double* v, double* z, cudaStream_t s);
void launch_cast_f64_f32(int n, const double* a, float* b, cudaStream_t s);
void launch_cast_f32_f64(int n, const float* a, double* b, cudaStream_t s);
void launch_copy_f64(int n, const double* a, double* b, cudaStream_t s);

// Arnoldi / vector kernels (FP64)
constexpr int kDotBlocks = 608;  // 4 x 152 SMs
// modified Gram-Schmidt of w against V[:, 0..nv-1]: h[i], *nrm2 = ||w||^2
void launch_mgs(int n, const double* V, long long ldv, int nv, double* w, double* h, double* nrm2, double* pa,
                double* pb, cudaStream_t s, const std::function<void()>& steps_begin = {},
                const std::function<void()>& steps_end = {});
// rev: traverse the vectors backwards (the streaming Arnoldi alternates
// directions between passes; 1 after a launch_mgs whose last step ran forwards)
void launch_scale_by_norm(int n, const double* w, const double* nrm2, double* v, cudaStream_t s, int rev = 0);
// the same modified Gram-Schmidt pass plus the scaling, as one cooperative
// grid of nb blocks with w in shared memory (nb from arnoldi_coop_blocks; part:
// (nv + 1) * nb doubles)
int arnoldi_coop_blocks(int n);
void launch_arnoldi_coop(int nb, int n, const double* V, long long ldv, int nv, const double* w, double* h,
                         double* nrm2, double* part, double* vout, cudaStream_t s);
void launch_vcomb(int n, const double* Z, long long ldz, int nv, const double* y, double* x, cudaStream_t s);
void launch_norm2(int n, const double* x, double* partial, double* out, cudaStream_t s);
void launch_block_resid(int N, int nc, const int* const* brp, const int* const* bci, const double* const* bv,
                        const double* const* dtab, const IOSlots* io, double* r, cudaStream_t s);
void launch_saxpy_vec(int n, double a, const double* x, double* y, cudaStream_t s);
void launch_lincomb(int n, double a, const double* x, double b, const double* y, double* out, cudaStream_t s);

}  // namespace mgd
