// mgd_host.cu -- host orchestration of the solver: AMG hierarchy setup on the
// device (Section 3.1), batched V-cycle plans and their autotuner, the block
// preconditioners (Sections 3.1, 3.3-3.6), right-preconditioned FGMRES(m)
// (Section 2 and the stopping rule of Section 4) and the C ABI.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <cstdlib>
#include <fstream>
#include <map>
#include <sstream>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include <unistd.h>

#include "../../include/mgdamg.h"
#include "mgd_internal.cuh"

namespace mgd {

long long g_kernel_launches = 0;
thread_local cudaMemPool_t tl_pool = nullptr;
thread_local bool tl_pdl = false;
thread_local cudaStream_t tl_stream = nullptr;
thread_local ScratchRegion* tl_region = nullptr;

enum OpKind { OP_A = 0, OP_CE = 1, OP_CG = 2, OP_SG = 3, OP_SI = 4, OP_AC = 5, OP_MONO = 6 };

// ------------------------------------------------------------------ profiler
// CUDA-event timing of selected kernel classes.  Stream launches are
// bracketed by events recorded on the stream; launches inside a captured graph
// are bracketed by event-record nodes of that graph.  Pending events are
// harvested (converted to durations) at the solver's host synchronisation
// points, so a graph replayed once per FGMRES iteration is timed every time.
struct Profiler {
  bool on = false;
  unsigned mask = 0;       // classes to record
  bool capturing = false;  // inside stream capture: record graph event nodes
  bool suppress = false;   // inside a conditional node's body: no event nodes allowed
  struct Pair {
    int cls;
    cudaEvent_t a, b;
    double bytes;
    int detail;   // second class (per level and phase), -1 if none
    double fp64;  // algorithmic FP64 lane operations of the bracketed launches
  };
  static constexpr int kClasses = 512;
  std::vector<Pair> pending, graph_pairs;
  bool graph_replayed = false;
  std::vector<cudaEvent_t> pool;
  long long n[kClasses] = {0};
  double ms[kClasses] = {0}, bytes[kClasses] = {0}, fp64[kClasses] = {0};
  int next_detail = -1;  // detail class of the next begin()
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    MGD_CUDA(cudaEventCreate(&e));
    return e;
  }
  void record(cudaEvent_t e, cudaStream_t s) {
    if (capturing) MGD_CUDA(cudaEventRecordWithFlags(e, s, cudaEventRecordExternal));
    else MGD_CUDA(cudaEventRecord(e, s));
  }
  int begin(cudaStream_t s, int cls) {
    if (!on || suppress || !(mask & (1u << cls))) {
      next_detail = -1;
      return -1;
    }
    cudaEvent_t a = get();
    record(a, s);
    auto& v = capturing ? graph_pairs : pending;
    v.push_back({cls, a, nullptr, 0.0, next_detail, 0.0});
    next_detail = -1;
    return (int)v.size() - 1;
  }
  void end(int id, int cls, double by, cudaStream_t s, double f64 = 0.0) {
    if (id < 0) return;
    cudaEvent_t b = get();
    record(b, s);
    auto& v = capturing ? graph_pairs : pending;
    v[id].cls = cls;
    v[id].b = b;
    v[id].bytes = by;
    v[id].fp64 = f64;
  }
  void add(const Pair& p) {
    float e = 0;
    MGD_CUDA(cudaEventElapsedTime(&e, p.a, p.b));
    n[p.cls]++;
    ms[p.cls] += e;
    bytes[p.cls] += p.bytes;
    fp64[p.cls] += p.fp64;
    if (p.detail >= 0 && p.detail < kClasses) {
      n[p.detail]++;
      ms[p.detail] += e;
      bytes[p.detail] += p.bytes;
      fp64[p.detail] += p.fp64;
    }
  }
  // call after the stream has been synchronised
  void harvest() {
    for (auto& p : pending) {
      if (p.b) add(p);
      pool.push_back(p.a);
      if (p.b) pool.push_back(p.b);
    }
    pending.clear();
    if (graph_replayed)
      for (auto& p : graph_pairs)
        if (p.b) add(p);
    graph_replayed = false;
  }
  void drop_graph_pairs() {
    for (auto& p : graph_pairs) {
      pool.push_back(p.a);
      if (p.b) pool.push_back(p.b);
    }
    graph_pairs.clear();
  }
  void reset() {
    for (auto& p : pending) {
      pool.push_back(p.a);
      if (p.b) pool.push_back(p.b);
    }
    pending.clear();
    graph_replayed = false;
    for (int k = 0; k < kClasses; ++k) {
      n[k] = 0;
      ms[k] = bytes[k] = fp64[k] = 0;
    }
  }
  ~Profiler() {
    for (auto& p : pending) {
      cudaEventDestroy(p.a);
      if (p.b) cudaEventDestroy(p.b);
    }
    for (auto& p : graph_pairs) {
      cudaEventDestroy(p.a);
      if (p.b) cudaEventDestroy(p.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

// ------------------------------------------------------------------ options
struct Opts {
  mgd_opts o;
};

// ------------------------------------------------------------------ hierarchy
struct Level {
  Csr A;
  float* v32 = nullptr;
  double* vpre = nullptr;   // A D^-1 values (CSR order)
  float* vpre32 = nullptr;
  double* atvpre = nullptr; // A^T D^-1 values
  float* atvpre32 = nullptr;
  Sell sell;
  double* dinv = nullptr;
  float* dinv32 = nullptr;
  Csr P, R;
  float *pv32 = nullptr, *rv32 = nullptr;
  Csr AT;
  float* atv32 = nullptr;
  Sell sellT;
  signed char* CF = nullptr;
  int nc = 0;
  void *b = nullptr, *x = nullptr, *xt = nullptr, *r = nullptr;
  // Gauss-Seidel order (smoother 1, levels with a C/F split)
  int nk = 0;
  int* key = nullptr;
  int* perm = nullptr;
  int* koff = nullptr;
  std::vector<int> koff_h;
  double* gdinv = nullptr;
  float* gdinv32 = nullptr;
  Sell gsell;  // rows in sweep order (forward operator)
};

struct Hier {
  std::vector<Level> L;
  bool coarse_lu = false;
  double* cinv = nullptr;
  double* cinvT = nullptr;
  int cn = 0;
  int* active = nullptr;  // device flag of a device-controlled inverse (nullptr: none)
  int nlev() const { return (int)L.size(); }
};

// host wall time per setup phase, summed over all hierarchy builds (worker
// threads add concurrently, so the hierarchy phases can sum past wall time)
enum SetupPhase {
  SP_STRENGTH = 0, SP_PMIS, SP_INTERP, SP_TRANSPOSE, SP_AP, SP_RAP, SP_FINALIZE, SP_COARSE,
  SP_VALIDATE, SP_BLOCKS, SP_HIERARCHIES, SP_PCTL, SP_PROGRAM, SP_KRYLOV, SP_COLOUR, SP_H2D, SP_RELEASE,
  SP_COUNT = 17
};
struct PhaseClock {
  std::mutex mu;
  double ms[SP_COUNT] = {0};
  void add(int ph, double v) {
    std::lock_guard<std::mutex> lk(mu);
    ms[ph] += v;
  }
  void reset() {
    std::lock_guard<std::mutex> lk(mu);
    for (double& x : ms) x = 0;
  }
};
struct PhaseTimer {
  PhaseClock* clk;
  int ph;
  std::chrono::steady_clock::time_point t0;
  PhaseTimer(PhaseClock* c, int p) : clk(c), ph(p), t0(std::chrono::steady_clock::now()) {}
  void stop() {
    if (!clk) return;
    clk->add(ph, std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count());
    clk = nullptr;
  }
  ~PhaseTimer() { stop(); }
};

struct SetupCtx {
  Arena* arena;
  cudaStream_t s;
  const mgd_opts* o;
  bool mixed;
  bool keepT;
  PhaseClock* clk;
};

static Csr csr_alloc(Arena& a, int n, int m, int nnz) {
  Csr c;
  c.n = n;
  c.m = m;
  c.nnz = nnz;
  c.rp = a.alloc<int>(n + 1);
  c.ci = a.alloc<int>(nnz);
  c.v = a.alloc<double>(nnz);
  return c;
}

static Csr csr_copy(Arena& a, const Csr& x, cudaStream_t s) {
  Csr c = csr_alloc(a, x.n, x.m, x.nnz);
  MGD_CUDA(cudaMemcpyAsync(c.rp, x.rp, sizeof(int) * (x.n + 1), cudaMemcpyDeviceToDevice, s));
  MGD_CUDA(cudaMemcpyAsync(c.ci, x.ci, sizeof(int) * x.nnz, cudaMemcpyDeviceToDevice, s));
  MGD_CUDA(cudaMemcpyAsync(c.v, x.v, sizeof(double) * x.nnz, cudaMemcpyDeviceToDevice, s));
  return c;
}

// C = X Y with the accumulation order of the Galerkin products (see setup_kernels.cu)
// C = X Y; C's arrays come from `keep` when given (a scratch that outlives C), else from the arena
static Csr spgemm(Arena& a, const Csr& X, const Csr& Y, cudaStream_t s, Scratch* keep = nullptr) {
  Scratch sc(s, a.pool);
  int n = X.n;
  int* ub = sc.alloc<int>(n);
  launch_spgemm_ub(n, X.rp, X.ci, Y.rp, ub, s);
  long long* off = sc.alloc<long long>(n + 1);
  launch_offsets64(ub, off, n, s);
  long long total = 0;
  MGD_CUDA(cudaMemcpyAsync(&total, off + n, sizeof(long long), cudaMemcpyDeviceToHost, s));
  MGD_CUDA(cudaStreamSynchronize(s));
  int* tc = sc.alloc<int>(total);
  double* tv = sc.alloc<double>(total);
  int* cnt = sc.alloc<int>(n);
  int* work = sc.alloc<int>(2 * (size_t)n + 2);
  launch_spgemm_expand(n, X.rp, X.ci, X.v, Y.rp, Y.ci, Y.v, off, tc, tv, cnt, work, s, total);
  Csr C;
  C.n = n;
  C.m = Y.m;
  C.rp = keep ? keep->alloc<int>(n + 1) : a.alloc<int>(n + 1, false, s);
  exclusive_scan(cnt, C.rp, n, s);
  C.nnz = read_int(C.rp + n, s);
  C.ci = keep ? keep->alloc<int>(C.nnz) : a.alloc<int>(C.nnz, false, s);
  C.v = keep ? keep->alloc<double>(C.nnz) : a.alloc<double>(C.nnz, false, s);
  launch_spgemm_compact(n, off, tc, tv, C.rp, C.ci, C.v, s);
  return C;
}

static Csr transpose(Arena& a, const Csr& X, cudaStream_t s, Scratch* keep = nullptr) {
  Scratch sc(s);
  Csr T;
  T.n = X.m;
  T.m = X.n;
  T.nnz = X.nnz;
  const int m1 = std::max(X.m, 1);
  int* cnt = sc.alloc<int>(2 * (size_t)m1);  // column counts, then the fill cursors
  int* cur = cnt + m1;
  MGD_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * 2 * (size_t)m1, s));
  launch_transpose_count(X.nnz, X.ci, cnt, s);
  T.rp = keep ? keep->alloc<int>(T.n + 1) : a.alloc<int>(T.n + 1);
  exclusive_scan(cnt, T.rp, T.n, s);
  T.ci = keep ? keep->alloc<int>(T.nnz) : a.alloc<int>(T.nnz);
  T.v = keep ? keep->alloc<double>(T.nnz) : a.alloc<double>(T.nnz);
  launch_transpose_fill(X.n, X.rp, X.ci, X.v, T.rp, cur, T.ci, T.v, s);
  launch_sort_rows(T.n, T.rp, T.ci, T.v, s);
  return T;
}

// SELL-32 copy of A in the V-cycle's precision only (FP32 values when mixed,
// else FP64); with dinv given, also A D^-1 in the same layout (vpre).
static Sell build_sell(Arena& a, const Csr& A, bool mixed, cudaStream_t s, const int* selfmap = nullptr,
                       const double* dinv = nullptr) {
  Scratch sc(s);
  Sell S;
  S.n = A.n;
  S.nslices = (A.n + 31) / 32;
  int* w = sc.alloc<int>(S.nslices);
  launch_sell_widths(A.n, A.rp, w, s);
  S.sptr = a.alloc<int>(S.nslices + 1);
  exclusive_scan(w, S.sptr, S.nslices, s);
  S.nstored = read_int(S.sptr + S.nslices, s);
  S.ci = a.alloc<int>(S.nstored);
  if (mixed) {
    S.v32 = a.alloc<float>(S.nstored);
    if (dinv) S.vpre32 = a.alloc<float>(S.nstored);
    launch_sell_fill(A.n, A.rp, A.ci, A.v, dinv, S.sptr, S.ci, S.v32, S.vpre32, s, selfmap);
  } else {
    S.v = a.alloc<double>(S.nstored);
    if (dinv) S.vpre = a.alloc<double>(S.nstored);
    launch_sell_fill(A.n, A.rp, A.ci, A.v, dinv, S.sptr, S.ci, S.v, S.vpre, s, selfmap);
  }
  return S;
}

static float* cast32(Arena& a, const double* x, int n, cudaStream_t s) {
  float* y = a.alloc<float>(n);
  launch_cast_f64_f32(n, x, y, s);
  return y;
}

// Gauss-Seidel order of a level (Section 3.1's C/F relaxation): colouring of
// the symmetrised graph, then sweep classes C(colour 0..), F(colour 0..) with
// the empty ones dropped, each class's rows listed in increasing order.
static void gs_order(Arena& ar, Level& lv, int level, unsigned long long seed, cudaStream_t s) {
  const int n = lv.A.n;
  Scratch tmp(s);
  // pattern of A^T, scratch only (rows unsorted: the colouring does not need order)
  const int nnz = lv.A.nnz;
  int* tcnt = tmp.alloc<int>(n);
  MGD_CUDA(cudaMemsetAsync(tcnt, 0, sizeof(int) * std::max(n, 1), s));
  launch_transpose_count(nnz, lv.A.ci, tcnt, s);
  int* trp = tmp.alloc<int>(n + 1);
  exclusive_scan(tcnt, trp, n, s);
  int* tci = tmp.alloc<int>(nnz);
  double* tv = tmp.alloc<double>(nnz);
  int* tcur = tmp.alloc<int>(n);
  MGD_CUDA(cudaMemsetAsync(tcur, 0, sizeof(int) * std::max(n, 1), s));
  launch_transpose_fill(n, lv.A.rp, lv.A.ci, lv.A.v, trp, tcur, tci, tv, s);
  Csr AT;
  AT.rp = trp;
  AT.ci = tci;
  double* w = tmp.alloc<double>(n);
  int* col = tmp.alloc<int>(n);
  int* nxt = tmp.alloc<int>(n);
  int* left = tmp.alloc<int>(1);
  launch_colour_init(n, seed, level, w, col, s);
  // rounds are idempotent once every point is coloured: check every second round
  for (int round = 0; round < n + 1; round += 2) {
    MGD_CUDA(cudaMemsetAsync(left, 0, sizeof(int), s));
    launch_colour_round(n, lv.A.rp, lv.A.ci, AT.rp, AT.ci, w, col, nxt, left, s);
    MGD_CUDA(cudaMemsetAsync(left, 0, sizeof(int), s));
    launch_colour_round(n, lv.A.rp, lv.A.ci, AT.rp, AT.ci, w, nxt, col, left, s);
    if (read_int(left, s) == 0) break;
  }
  int* mx = tmp.alloc<int>(1);
  MGD_CUDA(cudaMemsetAsync(mx, 0, sizeof(int), s));
  launch_colour_max(n, col, mx, s);
  const int ncol = read_int(mx, s) + 1;
  int* cnt = tmp.alloc<int>(2 * ncol);
  MGD_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * 2 * ncol, s));
  launch_key_count(n, col, lv.CF, ncol, cnt, s);
  std::vector<int> hc(2 * ncol), map(2 * ncol, -1);
  MGD_CUDA(cudaMemcpyAsync(hc.data(), cnt, sizeof(int) * 2 * ncol, cudaMemcpyDeviceToHost, s));
  MGD_CUDA(cudaStreamSynchronize(s));
  lv.koff_h.assign(1, 0);
  for (int k = 0; k < 2 * ncol; ++k)
    if (hc[k] > 0) {
      map[k] = (int)lv.koff_h.size() - 1;
      lv.koff_h.push_back(lv.koff_h.back() + hc[k]);
    }
  lv.nk = (int)lv.koff_h.size() - 1;
  int* dmap = tmp.alloc<int>(2 * ncol);
  MGD_CUDA(cudaMemcpyAsync(dmap, map.data(), sizeof(int) * 2 * ncol, cudaMemcpyHostToDevice, s));
  lv.koff = ar.alloc<int>(lv.nk + 1);
  MGD_CUDA(cudaMemcpyAsync(lv.koff, lv.koff_h.data(), sizeof(int) * (lv.nk + 1), cudaMemcpyHostToDevice, s));
  lv.key = ar.alloc<int>(n);
  launch_key_assign(n, col, lv.CF, ncol, dmap, lv.key, s);
  lv.perm = ar.alloc<int>(n);
  launch_key_perm(n, lv.nk, lv.key, lv.koff, lv.perm, s);
  MGD_CUDA(cudaStreamSynchronize(s));  // host vectors above go out of scope
}

// One coarsening pass on A (Section 3.1): strength, PMIS with the weight stream
// 1000 + lid, interpolation.  CF and P come from `keep` when given (a pass
// whose result is not kept as a level), else from the arena.  Returns false
// when the pass stalls (no C point, or all C).
struct Pass {
  signed char* CF = nullptr;
  int nc = 0;
  Csr P;
};
static bool coarsen_pass(SetupCtx& sc, const Csr& A, int lid, Scratch* keep, Pass& out) {
  Arena& ar = *sc.arena;
  cudaStream_t s = sc.s;
  const mgd_opts& o = *sc.o;
  const int n = A.n;
  Scratch tmp(s);
  PhaseTimer pt_str(sc.clk, SP_STRENGTH);
  uint8_t* S = tmp.alloc<uint8_t>(A.nnz);
  launch_strength(n, A.rp, A.ci, A.v, o.theta_str, S, s);
  int* cnt = tmp.alloc<int>(2 * (size_t)n);  // strong counts, then the fill cursors
  int* cur = cnt + n;
  MGD_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * 2 * (size_t)n, s));
  launch_count_st(n, A.rp, A.ci, S, cnt, s);
  int* strp = tmp.alloc<int>(n + 1);
  exclusive_scan(cnt, strp, n, s);
  int* stci = tmp.alloc<int>(A.nnz);  // at most every entry is strong: no read-back of the count
  launch_fill_st(n, A.rp, A.ci, S, strp, cur, stci, s);
  pt_str.stop();
  PhaseTimer pt_pmis(sc.clk, SP_PMIS);
  double* w = tmp.alloc<double>(n);
  signed char* CF = keep ? keep->alloc<signed char>(n) : ar.alloc<signed char>(n);
  launch_pmis_init(n, A.rp, S, cnt, o.seed, lid, w, CF, s);
  uint8_t* newc = tmp.alloc<uint8_t>(n);
  int* und = tmp.alloc<int>(1);
  // rounds are idempotent once every point is decided, so the undecided
  // count is read back only every second round
  for (int round = 0; round < n + 1; round += 2) {
    launch_pmis_round(n, A.rp, A.ci, S, strp, stci, w, CF, newc, und, s);
    launch_pmis_round(n, A.rp, A.ci, S, strp, stci, w, CF, newc, und, s);
    if (read_int(und, s) == 0) break;
  }
  pt_pmis.stop();
  PhaseTimer pt_int(sc.clk, SP_INTERP);
  int* pcnt = tmp.alloc<int>(n);
  int* isc = tmp.alloc<int>(n);
  launch_interp_count(n, A.rp, A.ci, S, CF, pcnt, isc, s);
  int* cidx = tmp.alloc<int>(n + 1);
  exclusive_scan(isc, cidx, n, s);
  // extended+i: upper bounds of the distance-two interpolatory sets, read
  // back with the coarse count in one synchronisation
  int* ub = nullptr;
  long long* off = nullptr;
  long long tot = 0;
  if (o.interp_type == 1) {
    ub = tmp.alloc<int>(n);
    launch_exti_ub(n, A.rp, A.ci, S, CF, pcnt, ub, s);
    off = tmp.alloc<long long>(n + 1);
    launch_offsets64(ub, off, n, s);
    MGD_CUDA(cudaMemcpyAsync(&tot, off + n, sizeof(long long), cudaMemcpyDeviceToHost, s));
  }
  int nc = read_int(cidx + n, s);
  if (nc == 0 || nc == n) return false;
  Csr P;
  P.n = n;
  P.m = nc;
  P.rp = keep ? keep->alloc<int>(n + 1) : ar.alloc<int>(n + 1);
  if (o.interp_type == 1) {  // extended+i: distance-two interpolatory sets
    int* list = tmp.alloc<int>(tot);
    int* len = tmp.alloc<int>(n);
    launch_exti_list(n, A.rp, A.ci, S, CF, off, list, len, s);
    exclusive_scan(len, P.rp, n, s);
    P.nnz = read_int(P.rp + n, s);
    P.ci = keep ? keep->alloc<int>(P.nnz) : ar.alloc<int>(P.nnz);
    P.v = keep ? keep->alloc<double>(P.nnz) : ar.alloc<double>(P.nnz);
    double* dg = tmp.alloc<double>(n);
    launch_diag_extract(n, A.rp, A.ci, A.v, dg, s);
    int* wi = tmp.alloc<int>((size_t)A.nnz + P.nnz);
    double* wd = tmp.alloc<double>((size_t)A.nnz + n);
    launch_exti_fill(n, A.nnz, A.rp, A.ci, A.v, S, CF, cidx, off, list, len, P.rp, P.nnz, P.ci, P.v, dg, wi, wd, s);
  } else {
    exclusive_scan(pcnt, P.rp, n, s);
    P.nnz = read_int(P.rp + n, s);
    P.ci = keep ? keep->alloc<int>(P.nnz) : ar.alloc<int>(P.nnz);
    P.v = keep ? keep->alloc<double>(P.nnz) : ar.alloc<double>(P.nnz);
    double* dg = tmp.alloc<double>(n);
    launch_diag_extract(n, A.rp, A.ci, A.v, dg, s);
    int* wi = tmp.alloc<int>((size_t)A.nnz + P.nnz);
    double* wd = tmp.alloc<double>((size_t)A.nnz + n);
    launch_interp_fill(n, A.nnz, A.rp, A.ci, A.v, S, CF, cidx, P.rp, P.nnz, P.ci, P.v, dg, wi, wd, s);
  }
  pt_int.stop();
  out.CF = CF;
  out.nc = nc;
  out.P = P;
  return true;
}

// Aggressive coarsening of level l (Section 3.1): a second pass, with the
// weight stream 1100 + l, on A1 = P1^T A P1 (not kept as a level) picks the
// final C points among the first pass's; P = P1 P2.  The first pass's C
// points that the second pass makes F become F.  A stalled second pass keeps
// the first pass.
static void aggressive_pass(SetupCtx& sc, const Csr& A, int l, Pass& pass) {
  Arena& ar = *sc.arena;
  cudaStream_t s = sc.s;
  const int n = A.n;
  Scratch ak(s, ar.pool);
  Csr R1 = transpose(ar, pass.P, s, &ak);
  Csr AP1 = spgemm(ar, A, pass.P, s, &ak);
  Csr A1 = spgemm(ar, R1, AP1, s, &ak);
  Pass p2;
  if (!coarsen_pass(sc, A1, 100 + l, &ak, p2)) return;
  Csr P = spgemm(ar, pass.P, p2.P, s);
  int* flag = ak.alloc<int>(n);
  int* cidx = ak.alloc<int>(n + 1);
  launch_cf_flag(n, pass.CF, flag, s);
  exclusive_scan(flag, cidx, n, s);
  launch_cf_compose(n, pass.CF, cidx, p2.CF, s);
  pass.P = P;
  pass.nc = p2.nc;
  MGD_CUDA(cudaStreamSynchronize(s));
}

// Section 3.1 setup: strength -> PMIS -> interpolation -> R = P^T -> A_c = R (A P),
// level by level until the coarsest criterion; then smoother diagonals,
// kernel layouts, FP32 copies and the coarsest dense inverse.
static void build_hierarchy(SetupCtx& sc, Hier& h, const Csr& A0) {
  Arena& ar = *sc.arena;
  cudaStream_t s = sc.s;
  const mgd_opts& o = *sc.o;
  h.L.clear();
  h.L.emplace_back();
  h.L[0].A = A0;
  for (int l = 0;; ++l) {
    Level& lv = h.L[l];
    int n = lv.A.n;
    if (n <= o.max_coarse || l == o.max_levels - 1) break;
    Pass pass;
    if (!coarsen_pass(sc, lv.A, l, nullptr, pass)) break;  // coarsening stalled: this level is the coarsest
    if (l < o.agg_levels) aggressive_pass(sc, lv.A, l, pass);
    lv.CF = pass.CF;
    lv.nc = pass.nc;
    if (o.smoother == 1) {
      PhaseTimer pt_col(sc.clk, SP_COLOUR);
      gs_order(ar, lv, l, o.seed, s);
    }
    Csr P = pass.P;
    lv.P = P;
    PhaseTimer pt_tr(sc.clk, SP_TRANSPOSE);
    lv.R = transpose(ar, P, s);
    pt_tr.stop();
    PhaseTimer pt_ap(sc.clk, SP_AP);
    Scratch apk(s, ar.pool);
    Csr AP = spgemm(ar, lv.A, P, s, &apk);
    pt_ap.stop();
    PhaseTimer pt_rap(sc.clk, SP_RAP);
    Csr Ac = spgemm(ar, lv.R, AP, s);
    pt_rap.stop();
    h.L.emplace_back();
    h.L.back().A = Ac;
  }
  // finalize levels
  PhaseTimer pt_fin(sc.clk, SP_FINALIZE);
  for (int l = 0; l < h.nlev(); ++l) {
    Level& lv = h.L[l];
    int n = lv.A.n;
    lv.dinv = ar.alloc<double>(n);
    if (sc.mixed) lv.dinv32 = ar.alloc<float>(n);
    launch_l1_dinv(n, lv.A.rp, lv.A.v, lv.dinv, s, lv.dinv32);
    if (lv.nk > 0) {
      lv.gdinv = ar.alloc<double>(n);
      launch_diag_inv(n, lv.A.rp, lv.A.ci, lv.A.v, lv.gdinv, s);
      if (sc.mixed) lv.gdinv32 = cast32(ar, lv.gdinv, n, s);
      Scratch ps(s);
      Csr Ap;
      Ap.n = n;
      Ap.m = lv.A.m;
      Ap.nnz = lv.A.nnz;
      int* len = ps.alloc<int>(n);
      launch_perm_row_len(n, lv.perm, lv.A.rp, len, s);
      Ap.rp = ps.alloc<int>(n + 1);
      exclusive_scan(len, Ap.rp, n, s);
      Ap.ci = ps.alloc<int>(Ap.nnz);
      Ap.v = ps.alloc<double>(Ap.nnz);
      launch_perm_rows_fill(n, lv.perm, lv.A.rp, lv.A.ci, lv.A.v, Ap.rp, Ap.ci, Ap.v, s);
      lv.gsell = build_sell(ar, Ap, sc.mixed, s, lv.perm);
    }
    // A D^-1 feeds only the l1-Jacobi pre-smoothing.  The FP32 form keeps the
    // FP64 CSR values (Galerkin products, coarsest inverse) and builds every
    // kernel array in FP32 straight from them: each FP32 value is the FP64
    // value (or the FP64 product a_ij d_j) rounded once.
    const bool jac = lv.nk == 0;
    const double* pre = jac ? lv.dinv : nullptr;
    lv.sell = build_sell(ar, lv.A, sc.mixed, s, nullptr, pre);
    if (sc.mixed) {
      lv.v32 = ar.alloc<float>(lv.A.nnz);
      if (jac) lv.vpre32 = ar.alloc<float>(lv.A.nnz);
      launch_colscale_f32(lv.A.nnz, lv.A.ci, lv.A.v, pre, lv.v32, lv.vpre32, s);
      if (l < h.nlev() - 1) {
        lv.pv32 = cast32(ar, lv.P.v, lv.P.nnz, s);
        lv.rv32 = cast32(ar, lv.R.v, lv.R.nnz, s);
      }
    } else if (jac) {
      lv.vpre = ar.alloc<double>(lv.A.nnz);
      launch_colscale(lv.A.nnz, lv.A.ci, lv.A.v, lv.dinv, lv.vpre, s);
    }
    if (sc.keepT) {
      lv.AT = transpose(ar, lv.A, s);
      lv.sellT = build_sell(ar, lv.AT, sc.mixed, s, nullptr, pre);
      if (sc.mixed) {
        lv.atv32 = ar.alloc<float>(lv.AT.nnz);
        if (jac) lv.atvpre32 = ar.alloc<float>(lv.AT.nnz);
        launch_colscale_f32(lv.AT.nnz, lv.AT.ci, lv.AT.v, pre, lv.atv32, lv.atvpre32, s);
      } else if (jac) {
        lv.atvpre = ar.alloc<double>(lv.AT.nnz);
        launch_colscale(lv.AT.nnz, lv.AT.ci, lv.AT.v, lv.dinv, lv.atvpre, s);
      }
    }
    // the level's vectors b, xt, (x,) r in one zeroed block, each 256-byte aligned;
    // Gauss-Seidel levels smooth in place: the level's output is xt itself
    size_t es = sc.mixed ? sizeof(float) : sizeof(double);
    const size_t vb = (es * n + 255) & ~(size_t)255;
    const int nvec = lv.nk > 0 ? 3 : 4;
    char* vecs = ar.alloc<char>(vb * nvec);
    MGD_CUDA(cudaMemsetAsync(vecs, 0, vb * nvec, s));
    lv.b = vecs;
    lv.xt = vecs + vb;
    lv.x = lv.nk > 0 ? lv.xt : vecs + 2 * vb;
    lv.r = vecs + (nvec - 1) * vb;
  }
  MGD_CUDA(cudaStreamSynchronize(s));
  pt_fin.stop();
  PhaseTimer pt_co(sc.clk, SP_COARSE);
  Level& last = h.L.back();
  if (last.A.n <= o.max_coarse) {
    int n = last.A.n;
    Scratch tmp(s);
    double* a = tmp.alloc<double>((size_t)n * n);
    int* piv = tmp.alloc<int>(n);
    int* st = tmp.alloc<int>(1);
    MGD_CUDA(cudaMemsetAsync(st, 0, sizeof(int), s));
    h.cinv = ar.alloc<double>((size_t)n * n);
    h.cinvT = ar.alloc<double>((size_t)n * n);
    launch_densify(n, last.A.rp, last.A.ci, last.A.v, a, s);
    launch_dense_inverse(n, a, piv, h.cinv, h.cinvT, st, s);
    if (read_int(st, s) != 0) throw Error{MGD_ESINGULAR, "zero pivot in the coarsest-level elimination"};
    h.coarse_lu = true;
    h.cn = n;
  }
}

// ------------------------------------------------------------------ batched V-cycle plans
template <typename T>
struct VBatch {
  std::vector<Hier*> hs;
  int depth = 0;
  struct LP {
    LDesc<T>* d_down = nullptr;
    int ndown = 0, maxn = 0, maxnc = 0;
    LDesc<T>* d_clu = nullptr;
    int nclu = 0, maxcn = 0;
    LDesc<T>* d_cjac = nullptr;
    int ncjac = 0, maxcj = 0;
    int fmtA = FMT_SELL, fmtR = FMT_CSR4, fmtP = FMT_CSR1;
    double bytes_pre = 0, bytes_post = 0, bytes_restrict = 0, bytes_prolong = 0, bytes_coarse = 0, bytes_jac = 0;
    double bytes_post_cj = 0;  // post-smoothing of the stalled coarsest levels
    // algorithmic FP64 lane operations (one per nonzero, two per row; FP64
    // values and l1-Jacobi levels only): the FP64 issue roofline of level 0
    double fp64_pre = 0, fp64_post = 0, fp64_cj = 0;
    // Gauss-Seidel levels: sweep steps and, per step, the largest class over the subsystems
    bool gs = false;
    int nkmax = 0, fmtGS = FMT_CSR4;  // sweep layout; SELL only where the sweep-ordered copy exists
    bool gs_sell = false;
    std::vector<int> seg_pre, seg_post;
  };
  std::vector<LP> plan, planT;
  double bytes_total = 0;
  // fused coarse-level kernel: levels >= tail_level of every subsystem in one
  // cluster launch (tail_level >= depth: not used)
  int tail_level = 1 << 20;
  int tail_cs = 8;
  TailSub<T>* d_tail = nullptr;
  TailSub<T>* d_tailT = nullptr;
  int ntail = 0;
  double tail_bytes = 0;
};

template <typename T>
static const T* pick(const double* d, const float* f);
template <>
const double* pick<double>(const double* d, const float*) {
  return d;
}
template <>
const float* pick<float>(const double*, const float* f) {
  return f;
}

template <typename T>
static LDesc<T> make_desc(Hier& h, int l, bool trans) {
  Level& lv = h.L[l];
  LDesc<T> d;
  memset(&d, 0, sizeof(d));
  d.n = lv.A.n;
  d.nc = lv.nc;
  const Csr& A = trans ? lv.AT : lv.A;
  const Sell& S = trans ? lv.sellT : lv.sell;
  d.rp = A.rp;
  d.ci = A.ci;
  d.v = pick<T>(A.v, trans ? lv.atv32 : lv.v32);
  d.sptr = S.sptr;
  d.sci = S.ci;
  d.sv = pick<T>(S.v, S.v32);
  d.vpre = trans ? pick<T>(lv.atvpre, lv.atvpre32) : pick<T>(lv.vpre, lv.vpre32);
  d.svpre = pick<T>(S.vpre, S.vpre32);
  d.dinv = pick<T>(lv.dinv, lv.dinv32);
  if (l < h.nlev() - 1) {
    d.prp = lv.P.rp;
    d.pci = lv.P.ci;
    d.pv = pick<T>(lv.P.v, lv.pv32);
    d.rrp = lv.R.rp;
    d.rci = lv.R.ci;
    d.rv = pick<T>(lv.R.v, lv.rv32);
    d.bc = (T*)h.L[l + 1].b;
    d.xc = (T*)h.L[l + 1].x;
  }
  d.b = (T*)lv.b;
  d.x = (T*)lv.x;
  d.xt = (T*)lv.xt;
  d.r = (T*)lv.r;
  d.cinv = trans ? h.cinvT : h.cinv;
  d.cn = h.cn;
  d.active = trans ? nullptr : h.active;
  d.nk = lv.nk;
  d.key = lv.key;
  d.perm = lv.perm;
  d.koff = lv.koff;
  d.gdinv = pick<T>(lv.gdinv, lv.gdinv32);
  if (!trans) {
    d.gsptr = lv.gsell.sptr;
    d.gsci = lv.gsell.ci;
    d.gsv = pick<T>(lv.gsell.v, lv.gsell.v32);
  }
  return d;
}

static double sp_bytes(long long nnz, long long rows, int sv) { return (double)nnz * (sv + 4) + 4.0 * (rows + 1); }

template <typename T>
static void build_plan(Arena& ar, VBatch<T>& vb, bool trans, cudaStream_t s) {
  auto& plan = trans ? vb.planT : vb.plan;
  vb.depth = 0;
  for (Hier* h : vb.hs) vb.depth = std::max(vb.depth, h->nlev());
  plan.assign(vb.depth, typename VBatch<T>::LP());
  const int sv = sizeof(T);
  double total = 0;
  for (int l = 0; l < vb.depth; ++l) {
    auto& lp = plan[l];
    std::vector<LDesc<T>> down, clu, cjac;
    for (Hier* h : vb.hs) {
      if (l >= h->nlev()) continue;
      Level& lv = h->L[l];
      LDesc<T> d = make_desc<T>(*h, l, trans);
      long long n = lv.A.n, nnz = lv.A.nnz;
      if (l < h->nlev() - 1) {
        down.push_back(d);
        lp.maxn = std::max<int>(lp.maxn, (int)n);
        lp.maxnc = std::max(lp.maxnc, lv.nc);
        if (lv.nk > 0) {
          // first sweep (key, b, 1/a_ii in; xt out), the other sweeps (rows once, perm,
          // b, 1/a_ii, xt read and written), the residual; up: every sweep
          if (!lp.gs) {
            lp.gs_sell = !trans;
            lp.fmtGS = lp.gs_sell ? FMT_SELL : FMT_CSR4;
          }
          lp.gs = true;
          lp.nkmax = std::max(lp.nkmax, lv.nk);
          if ((int)lp.seg_pre.size() < lv.nk) {
            lp.seg_pre.resize(lv.nk, 0);
            lp.seg_post.resize(lv.nk, 0);
          }
          for (int k = 0; k < lv.nk; ++k) {
            int c = lv.koff_h[k + 1] - lv.koff_h[k];
            lp.seg_pre[k] = std::max(lp.seg_pre[k], c);
            lp.seg_post[lv.nk - 1 - k] = std::max(lp.seg_post[lv.nk - 1 - k], c);
          }
          lp.bytes_pre += (4.0 + 3.0 * sv) * n + sp_bytes(nnz, n, sv) + (4.0 + 4.0 * sv) * n +
                          sp_bytes(nnz, n, sv) + 3.0 * sv * n;
          lp.bytes_post += sp_bytes(nnz, n, sv) + (4.0 + 4.0 * sv) * n;
        } else {
          lp.bytes_pre += sp_bytes(nnz, n, sv) + 4.0 * sv * n;
          lp.bytes_post += sp_bytes(nnz, n, sv) + 4.0 * sv * n;
          if (sv == 8) {  // k_pre: a multiply-add per nonzero, xt = D^-1 b, r = b - s; k_post likewise
            lp.fp64_pre += (double)nnz + 2.0 * n;
            lp.fp64_post += (double)nnz + 2.0 * n;
          }
        }
        lp.bytes_restrict += sp_bytes(lv.R.nnz, lv.nc, sv) + (double)sv * (n + lv.nc);
        lp.bytes_prolong += sp_bytes(lv.P.nnz, n, sv) + (double)sv * (lv.nc + 2 * n);
      } else if (h->coarse_lu) {
        clu.push_back(d);
        lp.maxcn = std::max(lp.maxcn, h->cn);
        lp.bytes_coarse += 8.0 * h->cn * h->cn + 2.0 * sv * h->cn;
      } else {
        cjac.push_back(d);
        lp.maxcj = std::max<int>(lp.maxcj, (int)n);
        lp.bytes_jac += 3.0 * sv * n;
        lp.bytes_post_cj += sp_bytes(nnz, n, sv) + 4.0 * sv * n;
        if (sv == 8) lp.fp64_cj += (double)nnz + 3.0 * n;
      }
    }
    auto upload = [&](std::vector<LDesc<T>>& v, LDesc<T>*& dst) {
      if (v.empty()) return;
      dst = ar.alloc<LDesc<T>>(v.size());
      MGD_CUDA(cudaMemcpyAsync(dst, v.data(), sizeof(LDesc<T>) * v.size(), cudaMemcpyHostToDevice, s));
    };
    upload(down, lp.d_down);
    upload(clu, lp.d_clu);
    upload(cjac, lp.d_cjac);
    lp.ndown = (int)down.size();
    lp.nclu = (int)clu.size();
    lp.ncjac = (int)cjac.size();
    total += lp.bytes_pre + lp.bytes_post + lp.bytes_restrict + lp.bytes_prolong + lp.bytes_coarse + lp.bytes_jac +
             lp.bytes_post_cj;
  }
  if (!trans) vb.bytes_total = total;
  MGD_CUDA(cudaStreamSynchronize(s));  // host vectors above go out of scope
}

// Gauss-Seidel smoothing of one level of a batch: down = first sweep from
// zero, sweeps 1.., residual; up = the sweeps in the opposite order
template <typename T>
static void run_gs_down(const typename VBatch<T>::LP& lp, cudaStream_t s) {
  launch_gs_first<T>(lp.d_down, lp.ndown, lp.maxn, s);
  for (int t = 1; t < lp.nkmax; ++t) launch_gs_sweep<T>(lp.fmtGS, lp.d_down, lp.ndown, lp.seg_pre[t], t, 0, s);
  launch_gs_resid<T>(lp.fmtA, lp.d_down, lp.ndown, lp.maxn, s);
}
template <typename T>
static void run_gs_up(const typename VBatch<T>::LP& lp, cudaStream_t s) {
  for (int t = 0; t < lp.nkmax; ++t) launch_gs_sweep<T>(lp.fmtGS, lp.d_down, lp.ndown, lp.seg_post[t], t, 1, s);
}

template <typename T>
static void run_vbatch(VBatch<T>& vb, bool trans, cudaStream_t s, Profiler& prof) {
  auto& plan = trans ? vb.planT : vb.plan;
  const bool tail = vb.tail_level < vb.depth && vb.ntail > 0;
  const int ltop = tail ? vb.tail_level : vb.depth;  // levels run with per-level launches
  for (int l = 0; l < ltop; ++l) {
    auto& lp = plan[l];
    if (lp.ndown) {
      prof.next_detail = 16 + 4 * l + 0;
      int id = prof.begin(s, l == 0 ? 0 : 1);
      if (lp.gs) run_gs_down<T>(lp, s);
      else launch_phase<T>(PH_PRE, lp.fmtA, lp.fmtR, lp.d_down, lp.ndown, lp.maxn, s);
      prof.end(id, l == 0 ? 0 : 1, lp.bytes_pre, s, lp.gs ? 0.0 : lp.fp64_pre);
      prof.next_detail = 16 + 4 * l + 1;
      id = prof.begin(s, 1);
      launch_phase<T>(PH_RESTRICT, lp.fmtA, lp.fmtR, lp.d_down, lp.ndown, lp.maxnc, s);
      prof.end(id, 1, lp.bytes_restrict, s);
    }
    if (lp.nclu) {
      prof.next_detail = 400 + l;
      int id = prof.begin(s, 1);
      launch_phase<T>(PH_COARSE, lp.fmtA, lp.fmtR, lp.d_clu, lp.nclu, lp.maxcn, s);
      prof.end(id, 1, lp.bytes_coarse, s);
    }
    if (lp.ncjac) {
      prof.next_detail = 400 + l;
      int id = prof.begin(s, l == 0 ? 0 : 1);
      launch_phase<T>(PH_JAC1, lp.fmtA, lp.fmtR, lp.d_cjac, lp.ncjac, lp.maxcj, s);
      launch_phase<T>(PH_POST, lp.fmtA, lp.fmtR, lp.d_cjac, lp.ncjac, lp.maxcj, s);
      prof.end(id, l == 0 ? 0 : 1, lp.bytes_jac + lp.bytes_post_cj, s, lp.fp64_cj);
    }
  }
  if (tail) {
    prof.next_detail = 15;
    int id = prof.begin(s, 1);
    launch_vtail<T>(trans ? vb.d_tailT : vb.d_tail, vb.ntail, vb.tail_cs, s);
    prof.end(id, 1, vb.tail_bytes, s);
  }
  for (int l = std::min(vb.depth - 2, ltop - 1); l >= 0; --l) {
    auto& lp = plan[l];
    if (!lp.ndown) continue;
    prof.next_detail = 16 + 4 * l + 2;
    int id = prof.begin(s, 1);
    launch_phase<T>(PH_PROLONG, lp.fmtA, lp.fmtP, lp.d_down, lp.ndown, lp.maxn, s);
    prof.end(id, 1, lp.bytes_prolong, s);
    prof.next_detail = 16 + 4 * l + 3;
    id = prof.begin(s, l == 0 ? 0 : 1);
    if (lp.gs) run_gs_up<T>(lp, s);
    else launch_phase<T>(PH_POST, lp.fmtA, lp.fmtP, lp.d_down, lp.ndown, lp.maxn, s);
    prof.end(id, l == 0 ? 0 : 1, lp.bytes_post, s, lp.gs ? 0.0 : lp.fp64_post);
  }
}

// Descriptors of the fused coarse-level kernel for the first fused level Lt:
// every subsystem with more than Lt levels contributes its levels Lt..coarsest.
template <typename T>
static void build_tail(Arena& ar, VBatch<T>& vb, int Lt, bool keepT, cudaStream_t s) {
  vb.tail_level = Lt;
  vb.ntail = 0;
  vb.tail_bytes = 0;
  if (Lt >= vb.depth) return;
  for (int pass = 0; pass < (keepT ? 2 : 1); ++pass) {
    bool trans = pass == 1;
    std::vector<TailSub<T>> subs;
    std::vector<std::vector<LDesc<T>>> keep;
    for (Hier* h : vb.hs) {
      if (h->nlev() <= Lt) continue;
      std::vector<LDesc<T>> lv;
      for (int l = Lt; l < h->nlev(); ++l) lv.push_back(make_desc<T>(*h, l, trans));
      LDesc<T>* d = ar.alloc<LDesc<T>>(lv.size());
      MGD_CUDA(cudaMemcpyAsync(d, lv.data(), sizeof(LDesc<T>) * lv.size(), cudaMemcpyHostToDevice, s));
      keep.push_back(std::move(lv));
      subs.push_back(TailSub<T>{d, h->nlev() - Lt, h->coarse_lu ? 1 : 0});
    }
    TailSub<T>* dt = subs.empty() ? nullptr : ar.alloc<TailSub<T>>(subs.size());
    if (dt) MGD_CUDA(cudaMemcpyAsync(dt, subs.data(), sizeof(TailSub<T>) * subs.size(), cudaMemcpyHostToDevice, s));
    MGD_CUDA(cudaStreamSynchronize(s));
    (trans ? vb.d_tailT : vb.d_tail) = dt;
    vb.ntail = (int)subs.size();
  }
  for (int l = Lt; l < vb.depth; ++l) {
    auto& lp = vb.plan[l];
    vb.tail_bytes += lp.bytes_pre + lp.bytes_post + lp.bytes_restrict + lp.bytes_prolong + lp.bytes_coarse +
                     lp.bytes_jac + lp.bytes_post_cj;
  }
}

// Autotune the first fused level: time whole V-cycles with no fusion and with
// fusion from the first level whose largest row count is below each threshold.
template <typename T>
static void autotune_tail(Arena& ar, VBatch<T>& vb, bool keepT, bool graph, cudaStream_t s) {
  Profiler none;
  std::vector<int> cand{vb.depth};
  for (int thr : {4096, 16384, 65536, 262144}) {
    int Lt = vb.depth;
    for (int l = 1; l < vb.depth; ++l) {
      auto& lp = vb.plan[l];
      int rows = std::max(lp.maxn, std::max(lp.maxcn, lp.maxcj));
      if (rows <= thr) {
        Lt = l;
        break;
      }
    }
    if (std::find(cand.begin(), cand.end(), Lt) == cand.end()) cand.push_back(Lt);
  }
  std::vector<int> sizes{8};
  if (vtail_cluster_fits<T>(16)) sizes.push_back(16);
  cudaEvent_t e0, e1;
  MGD_CUDA(cudaEventCreate(&e0));
  MGD_CUDA(cudaEventCreate(&e1));
  // time five V-cycles the way the solve will run them: replayed from a
  // captured graph when the context replays graphs (launch costs differ)
  auto time_cycles = [&]() -> float {
    float ms = 0;
    if (graph) {
      cudaGraph_t g = nullptr;
      cudaGraphExec_t ge = nullptr;
      MGD_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      try {
        for (int r = 0; r < 5; ++r) run_vbatch<T>(vb, false, s, none);
      } catch (...) {
        cudaStreamEndCapture(s, &g);
        if (g) cudaGraphDestroy(g);
        throw;
      }
      MGD_CUDA(cudaStreamEndCapture(s, &g));
      MGD_CUDA(cudaGraphInstantiate(&ge, g, 0));
      cudaGraphDestroy(g);
      MGD_CUDA(cudaGraphLaunch(ge, s));
      MGD_CUDA(cudaEventRecord(e0, s));
      MGD_CUDA(cudaGraphLaunch(ge, s));
      MGD_CUDA(cudaGraphLaunch(ge, s));
      MGD_CUDA(cudaEventRecord(e1, s));
      MGD_CUDA(cudaEventSynchronize(e1));
      cudaGraphExecDestroy(ge);
      MGD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      return ms / 2;
    }
    run_vbatch<T>(vb, false, s, none);
    MGD_CUDA(cudaEventRecord(e0, s));
    for (int r = 0; r < 5; ++r) run_vbatch<T>(vb, false, s, none);
    MGD_CUDA(cudaEventRecord(e1, s));
    MGD_CUDA(cudaEventSynchronize(e1));
    MGD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    return ms;
  };
  int best_lt = vb.depth, best_cs = 8;
  float best = 1e30f;
  for (int Lt : cand) {
    for (int cs : sizes) {
      if (Lt >= vb.depth && cs != 8) continue;
      vb.tail_cs = cs;
      build_tail<T>(ar, vb, Lt, keepT, s);
      float ms = time_cycles();
      if (ms < best * 0.97f) {  // prefer fewer fused levels unless clearly faster
        best = ms;
        best_lt = Lt;
        best_cs = cs;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  vb.tail_cs = best_cs;
  build_tail<T>(ar, vb, best_lt, keepT, s);
}

// Autotuner: per level of a batch, time the operator phase (PRE) under each
// sparse layout and the transfer phases under each threads-per-row choice;
// keep the fastest.  Inputs are the level buffers (zero at setup).
template <typename T>
static void autotune(VBatch<T>& vb, bool trans, cudaStream_t s) {
  auto& plan = trans ? vb.planT : vb.plan;
  cudaEvent_t e0, e1;
  MGD_CUDA(cudaEventCreate(&e0));
  MGD_CUDA(cudaEventCreate(&e1));
  auto time_it = [&](auto fn) {
    fn();
    fn();
    MGD_CUDA(cudaEventRecord(e0, s));
    for (int r = 0; r < 6; ++r) fn();
    MGD_CUDA(cudaEventRecord(e1, s));
    MGD_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    MGD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    return ms;
  };
  const int candA[] = {FMT_SELL, FMT_SELL2, FMT_SELL4, FMT_CSR1, FMT_CSR2, FMT_CSR4, FMT_CSR8};
  const int candRP[] = {FMT_CSR1, FMT_CSR1X2, FMT_CSR1X4, FMT_CSR2, FMT_CSR4, FMT_CSR8};
  for (int l = 0; l < vb.depth; ++l) {
    auto& lp = plan[l];
    if (!lp.ndown) continue;
    float best = 1e30f;
    for (int f : candA) {
      float ms = time_it([&] {
        if (lp.gs) launch_gs_resid<T>(f, lp.d_down, lp.ndown, lp.maxn, s);
        else launch_phase<T>(PH_PRE, f, lp.fmtR, lp.d_down, lp.ndown, lp.maxn, s);
      });
      if (ms < best) {
        best = ms;
        lp.fmtA = f;
      }
    }
    if (lp.gs) {  // layout of the sweeps: time a whole down-smoothing
      best = 1e30f;
      int pick = lp.fmtGS;
      for (int f : candA) {
        if (f == FMT_SELL2 || f == FMT_SELL4 || (f == FMT_SELL && !lp.gs_sell)) continue;
        lp.fmtGS = f;
        float ms = time_it([&] { run_gs_down<T>(lp, s); });
        if (ms < best) {
          best = ms;
          pick = f;
        }
      }
      lp.fmtGS = pick;
    }
    best = 1e30f;
    for (int f : candRP) {
      float ms = time_it([&] { launch_phase<T>(PH_RESTRICT, lp.fmtA, f, lp.d_down, lp.ndown, lp.maxnc, s); });
      if (ms < best) {
        best = ms;
        lp.fmtR = f;
      }
    }
    best = 1e30f;
    for (int f : candRP) {
      float ms = time_it([&] { launch_phase<T>(PH_PROLONG, lp.fmtA, f, lp.d_down, lp.ndown, lp.maxn, s); });
      if (ms < best) {
        best = ms;
        lp.fmtP = f;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
}

// ------------------------------------------------------------------ block preconditioner
struct InvOp {
  int kind, comp;
  Csr A;               // operator (FP64)
  bool jacobi = false; // option #1
  bool accurate = false;  // option #3 in the forward apply (inner_mode)
  int count = 1;       // sweeps (#1) or V-cycles (#2)
  Hier h;
  double* jd = nullptr;  // 1/diag(A)
  float* jd32 = nullptr;
  void* b = nullptr;     // rhs (type T): level-0 b of the hierarchy, or own buffer for #1
  void* x = nullptr;     // output (type T)
  void* bsave = nullptr; // extra buffers for several cycles / sweeps
  void* xacc = nullptr;
  int n = 0;
  float* v32 = nullptr;
  void* d_jac = nullptr;   // JacDesc<T>: x = D^-1 b
  void* d_jac2 = nullptr;  // JacDesc<T>: xacc = D^-1 bsave (further sweeps)
};

struct Step {
  // CONSPROD: a CONSUME (descs, nd) fused with the PRODUCE after it (descs2, nd2)
  enum { PRODUCE, INVERT, CONSUME, BLOCKRESID, CONSPROD } type;
  void* descs = nullptr;  // device descriptors
  int nd = 0;
  void* descs2 = nullptr;
  int nd2 = 0;
  int len = 0;            // vector length of produce/consume
  int nterms = 0;         // PRODUCE: coupling terms over all descriptors
  std::vector<int> ops;   // INVERT
  int batch = -1;         // index into batches when batched
  double bytes = 0;
  // INVERT with a device-controlled loop (option #3 or several cycles)
  bool loop = false;
  void* inner = nullptr;       // InnerDesc<T>[nloop] (device)
  InnerCtl* ctl = nullptr;     // device loop state
  long long* total = nullptr;  // == ctl->total (device), per loop op
  int* any = nullptr;          // == ctl->any (device)
  std::vector<int> loop_ops;   // op ids in InnerDesc order
  int maxn = 0, guard = 0;
};

struct BlockData {
  int G = 0, N = 0, nc = 0;
  std::vector<Csr> Ab;              // diagonal blocks
  std::vector<double*> d;           // nc*nc coupling vectors (nullptr: absent/dropped)
  std::vector<int> dropped;
  std::vector<double*> diag;        // diag(A_a)
  std::vector<double*> p;           // PCTL p_a
  Csr Ac;
  double** d_dtab = nullptr;        // device copy of d
  int** d_brp = nullptr;
  int** d_bci = nullptr;
  double** d_bv = nullptr;
};

}  // namespace mgd

// ------------------------------------------------------------------ context
struct mgd_ctx {
  mgd_opts o;
  cudaStream_t s = nullptr;
  int device = 0;
  std::string err;
  mgd::Pool pool;
  mgd::Arena ar;
  bool ready = false;
  int kind = 0, G = 0, N = 0, n = 0, nnz = 0;
  mgd::Csr A;      // monolithic operator (FP64)
  mgd::Sell Asell;
  int fmtMono = mgd::FMT_SELL;
  mgd::Csr AT;
  mgd::Sell ATsell;
  mgd::BlockData bd;
  std::vector<mgd::InvOp> ops;
  std::vector<mgd::Step> steps, stepsT;
  std::vector<mgd::VBatch<double>> vb64;
  std::vector<mgd::VBatch<float>> vb32;
  mgd::IOSlots* io = nullptr;
  double *wEs = nullptr, *wIs = nullptr, *rfull = nullptr;
  double *t4a = nullptr, *t4b = nullptr;  // option #4 work vectors (N)
  // FGMRES storage
  double *V = nullptr, *Z = nullptr, *w = nullptr, *r = nullptr, *hbuf = nullptr, *partial = nullptr,
         *ybuf = nullptr, *xtmp = nullptr, *btmp = nullptr;
  double* hpin = nullptr;  // pinned host
  int m = 30;
  std::vector<double> hist;
  mgd::Profiler prof;
  cudaGraphExec_t graph = nullptr;
  bool graph_ok = false;
  bool capturing = false;            // run_program is being recorded into c->graph
  cudaStream_t s_body = nullptr;     // stream that records conditional-node bodies
  cudaStream_t s_copy[4] = {nullptr, nullptr, nullptr, nullptr};  // host-to-device copies of mgd_setup_host
  long long graph_kernels = 0;
  long long napply = 0, napplyT = 0; // preconditioner applies since setup (forward, transposed)
  int arn_nb = 0;                    // blocks of the cooperative Arnoldi grid (0: streaming kernels)
  mgd_stats st;
  int n_jacobi = 0;
  mgd::PhaseClock phases;
};

namespace mgd {

static bool mixed(const mgd_ctx* c) { return c->o.precision == 1; }

static PRef ABS(double* p) { return PRef{0, 0, p}; }
static PRef VIN(long long off) { return PRef{1, off, nullptr}; }
static PRef ZOUT(long long off) { return PRef{2, off, nullptr}; }
static PRef NUL() { return PRef{0, 0, nullptr}; }

template <typename T>
static void add_produce(mgd_ctx* c, std::vector<ProduceDesc<T>>& v, int op, PRef a,
                        std::vector<std::tuple<const double*, PRef, double>> terms) {
  ProduceDesc<T> d;
  memset(&d, 0, sizeof(d));
  d.dst = (T*)c->ops[op].b;
  d.a = a;
  d.nt = 0;
  for (auto& t : terms) {
    if (d.nt >= kMaxTerms) throw Error{MGD_EINVAL, "too many coupling terms"};
    d.d[d.nt] = std::get<0>(t);
    d.w[d.nt] = std::get<1>(t);
    d.s[d.nt] = std::get<2>(t);
    d.nt++;
  }
  v.push_back(d);
}

template <typename T>
static void add_consume(std::vector<ConsumeDesc<T>>& v, PRef dst, PRef base, double s, const void* x,
                        const double* dvec = nullptr) {
  ConsumeDesc<T> d;
  memset(&d, 0, sizeof(d));
  d.dst = dst;
  d.base = base;
  d.s = s;
  d.unit = s == 1.0 ? 1 : (s == -1.0 ? 2 : 0);
  d.x = (const T*)x;
  (void)dvec;
  v.push_back(d);
}

template <typename D>
static void* upload_vec(mgd_ctx* c, const std::vector<D>& v) {
  if (v.empty()) return nullptr;
  D* d = c->ar.alloc<D>(v.size());
  MGD_CUDA(cudaMemcpyAsync(d, v.data(), sizeof(D) * v.size(), cudaMemcpyHostToDevice, c->s));
  MGD_CUDA(cudaStreamSynchronize(c->s));
  return d;
}

template <typename T>
static void push_produce(mgd_ctx* c, std::vector<Step>& steps, std::vector<ProduceDesc<T>> v, int len) {
  Step st;
  st.type = Step::PRODUCE;
  st.nd = (int)v.size();
  st.len = len;
  st.descs = upload_vec(c, v);
  for (auto& d : v) {
    st.bytes += (double)len * (sizeof(T) + (d.a.slot || d.a.abs ? 8 : 0) + 16.0 * d.nt);
    st.nterms += d.nt;
  }
  steps.push_back(st);
}
template <typename T>
static void push_consume(mgd_ctx* c, std::vector<Step>& steps, std::vector<ConsumeDesc<T>> v, int len) {
  Step st;
  st.type = Step::CONSUME;
  st.nd = (int)v.size();
  st.len = len;
  st.descs = upload_vec(c, v);
  for (auto& d : v) st.bytes += (double)len * (sizeof(T) + 8 + (d.base.slot || d.base.abs ? 8 : 0));
  steps.push_back(st);
}
static void push_invert(std::vector<Step>& steps, std::vector<int> ops) {
  Step st;
  st.type = Step::INVERT;
  st.ops = ops;
  steps.push_back(st);
}

// ------------------------------------------------------------------ inverse operators
template <typename T>
static void finalize_op(mgd_ctx* c, InvOp& op, cudaStream_t st) {
  const size_t es = sizeof(T);
  op.n = op.A.n;
  if (op.jacobi) {
    op.jd = c->ar.alloc<double>(op.n);
    launch_diag_inv(op.n, op.A.rp, op.A.ci, op.A.v, op.jd, st);
    if (mixed(c)) {
      op.jd32 = cast32(c->ar, op.jd, op.n, st);
      op.v32 = cast32(c->ar, op.A.v, op.A.nnz, st);
    }
    op.b = c->ar.alloc<char>(es * op.n, true, st);
    op.x = c->ar.alloc<char>(es * op.n, true, st);
  } else {
    SetupCtx sc{&c->ar, st, &c->o, mixed(c), c->o.keep_transpose != 0, &c->phases};
    build_hierarchy(sc, op.h, op.A);
    op.b = op.h.L[0].b;
    op.x = op.h.L[0].x;
  }
  if (op.count > 1 || op.accurate) {
    op.bsave = c->ar.alloc<char>(es * op.n, true, st);
    op.xacc = c->ar.alloc<char>(es * op.n, true, st);
  }
  if (op.jacobi) {
    JacDesc<T> j1{(T*)op.x, (const T*)op.b, pick<T>(op.jd, op.jd32)};
    JacDesc<T> j2{(T*)op.xacc, (const T*)op.bsave, pick<T>(op.jd, op.jd32)};
    JacDesc<T>* d = c->ar.alloc<JacDesc<T>>(2);
    MGD_CUDA(cudaMemcpyAsync(d, &j1, sizeof(j1), cudaMemcpyHostToDevice, st));
    MGD_CUDA(cudaMemcpyAsync(d + 1, &j2, sizeof(j2), cudaMemcpyHostToDevice, st));
    op.d_jac = d;
    op.d_jac2 = d + 1;
  }
  MGD_CUDA(cudaStreamSynchronize(st));
}

// worker threads of the concurrent hierarchy setup: at most MGD_SETUP_THREADS,
// at most MGD_SETUP_OVERSUB per host core
#ifndef MGD_SETUP_THREADS
#define MGD_SETUP_THREADS 16
#endif
#ifndef MGD_SETUP_OVERSUB
#define MGD_SETUP_OVERSUB 1
#endif

// Setup of independent operators runs concurrently: each worker thread owns a
// CUDA stream and builds whole hierarchies, so the many small host round
// trips of one hierarchy (scan totals, PMIS rounds) overlap with the others.
template <typename T>
static void finalize_ops_parallel(mgd_ctx* c, size_t first, size_t last) {
  size_t nops = last - first;
  if (nops == 0) return;
  MGD_CUDA(cudaStreamSynchronize(c->s));
  unsigned hw = std::thread::hardware_concurrency();
  size_t nthreads = std::min<size_t>(
      nops, std::max<unsigned>(1u, std::min<unsigned>((hw ? hw : 4) * MGD_SETUP_OVERSUB, MGD_SETUP_THREADS)));
  if (nthreads <= 1) {
    for (size_t k = first; k < last; ++k) finalize_op<T>(c, c->ops[k], c->s);
    return;
  }
  std::atomic<size_t> next(first);
  std::vector<Error> errs;
  std::mutex emu;
  auto worker = [&]() {
    cudaStream_t st = nullptr;
    ScratchRegion* region = nullptr;
    try {
      MGD_CUDA(cudaSetDevice(c->device));
      MGD_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
      tl_pool = c->ar.pool;
      tl_stream = st;
      region = new ScratchRegion(st, c->ar.pool);
      tl_region = region;
      for (size_t k = next++; k < last; k = next++) finalize_op<T>(c, c->ops[k], st);
    } catch (const Error& e) {
      std::lock_guard<std::mutex> lk(emu);
      errs.push_back(e);
    } catch (const std::exception& e) {
      std::lock_guard<std::mutex> lk(emu);
      errs.push_back(Error{MGD_ECUDA, e.what()});
    }
    tl_region = nullptr;
    if (st) cudaStreamSynchronize(st);
    delete region;  // its chunks are freed on st, after everything issued there
    if (st) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
    tl_stream = nullptr;
  };
  std::vector<std::thread> th;
  for (size_t t = 0; t < nthreads; ++t) th.emplace_back(worker);
  for (auto& t : th) t.join();
  if (!errs.empty()) throw errs.front();
}

static int cycles_for(const mgd_opts& o, int kind, int comp, int G) {
  if (kind == OP_AC || kind == OP_MONO) return o.nvcyc_other;
  if (comp < G) return o.nvcyc_group;
  if (comp == G) return o.nvcyc_E;
  return o.nvcyc_I;
}

static double gamma_wd(mgd_ctx* c, const Csr& A) {
  Scratch sc(c->s);
  int* cnt = sc.alloc<int>(1);
  MGD_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int), c->s));
  launch_gamma_wd(A.n, A.rp, A.ci, A.v, c->o.theta_wd, cnt, c->s);
  return A.n ? (double)read_int(cnt, c->s) / A.n : 0.0;
}

static int add_op(mgd_ctx* c, int kind, int comp, Csr A) {
  InvOp op;
  op.kind = kind;
  op.comp = comp;
  op.A = A;
  op.jacobi = c->o.adaptive && kind != OP_MONO && gamma_wd(c, A) == 0.0;
  op.count = op.jacobi ? c->o.jacobi_sweeps : cycles_for(c->o, kind, comp, c->G);
  if (op.count < 1) op.count = 1;
  // Section 4: the Schur-type inverses, and the PCTL block inverses, to the inner accuracy
  op.accurate = c->o.inner_mode && !op.jacobi &&
                (kind == OP_CE || kind == OP_CG || kind == OP_SG || kind == OP_SI ||
                 (c->kind == MGD_PCTL && kind == OP_A));
  c->ops.push_back(op);
  return (int)c->ops.size() - 1;
}

static Csr diag_modified(mgd_ctx* c, const Csr& A, const double* x, const double* y, const double* z) {
  Csr M = csr_copy(c->ar, A, c->s);
  if (x && y) launch_diag_modify(M.n, M.rp, M.ci, M.v, x, y, z, c->s);
  return M;
}

// run option #1 / #2 for a list of operators (one batch when batched)
template <typename T>
static void run_invert(mgd_ctx* c, const Step& st, bool trans);

template <typename T>
std::vector<VBatch<T>>& batches(mgd_ctx* c);
template <>
std::vector<VBatch<double>>& batches<double>(mgd_ctx* c) {
  return c->vb64;
}
template <>
std::vector<VBatch<float>>& batches<float>(mgd_ctx* c) {
  return c->vb32;
}

template <typename T>
static void apply_jacobi_ops(mgd_ctx* c, const std::vector<int>& ids, bool trans) {
  // option #1: x = D^-1 b, then further sweeps x += D^-1 (b - A x).  D is
  // diagonal, so the transposed operator uses the same D; the residual of
  // further sweeps uses A^T in the transposed apply.
  for (int id : ids) {
    InvOp& op = c->ops[id];
    launch_jacobi<T>((const JacDesc<T>*)op.d_jac, 1, op.n, c->s);
    for (int k = 1; k < op.count; ++k) {
      const Csr& A = op.A;
      launch_residual<T>(FMT_CSR4, op.n, A.rp, A.ci, pick<T>(A.v, op.v32), nullptr, nullptr, nullptr,
                         (const T*)op.b, (const T*)op.x, (T*)op.bsave, c->s);
      launch_jacobi<T>((const JacDesc<T>*)op.d_jac2, 1, op.n, c->s);
      launch_axpy<T>(op.n, (T*)op.x, (const T*)op.xacc, c->s);
    }
    (void)trans;
  }
}

// The device-controlled loop of one INVERT step.  Eager: the host reads the
// control kernel's "some operator active" flag after every trip.  Under graph
// capture: a conditional while node whose body (V-cycle, update, residual,
// control) is recorded on a second stream; the control kernel sets the node's
// condition, so a replay runs exactly the trips the eager loop would.
template <typename T>
static void run_inner_loop(mgd_ctx* c, const Step& st, VBatch<T>& B) {
  const InnerDesc<T>* d = (const InnerDesc<T>*)st.inner;
  const int nd = (int)st.loop_ops.size();
  const cudaGraphConditionalHandle none = 0;
  launch_inner_begin<T>(d, nd, st.maxn, st.ctl, c->s);
  if (!c->capturing) {
    launch_inner_ctl<T>(d, nd, st.ctl, 1, 0, none, c->s);
    for (int trip = 0; trip < st.guard && read_int(st.any, c->s); ++trip) {
      run_vbatch<T>(B, false, c->s, c->prof);
      launch_inner_update<T>(d, nd, st.maxn, c->s);
      launch_inner_resid<T>(d, nd, st.maxn, st.ctl, c->s);
      launch_inner_ctl<T>(d, nd, st.ctl, 0, 0, none, c->s);
    }
    launch_inner_end<T>(d, nd, st.maxn, c->s);
    return;
  }
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  MGD_CUDA(cudaStreamGetCaptureInfo(c->s, &cs, nullptr, &g, nullptr, nullptr, nullptr));
  cudaGraphConditionalHandle h;
  MGD_CUDA(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
  launch_inner_ctl<T>(d, nd, st.ctl, 1, 1, h, c->s);
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  MGD_CUDA(cudaStreamGetCaptureInfo(c->s, &cs, nullptr, &g, &deps, nullptr, &ndeps));
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  MGD_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  MGD_CUDA(cudaStreamUpdateCaptureDependencies(c->s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  // body nodes: kernels only (no event nodes, no programmatic edges)
  const bool pdl = tl_pdl;
  tl_pdl = false;
  c->prof.suppress = true;
  MGD_CUDA(cudaStreamBeginCaptureToGraph(c->s_body, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  cudaGraph_t recorded = nullptr;
  try {
    run_vbatch<T>(B, false, c->s_body, c->prof);
    launch_inner_update<T>(d, nd, st.maxn, c->s_body);
    launch_inner_resid<T>(d, nd, st.maxn, st.ctl, c->s_body);
    launch_inner_ctl<T>(d, nd, st.ctl, 0, 1, h, c->s_body);
  } catch (...) {
    cudaStreamEndCapture(c->s_body, &recorded);
    c->prof.suppress = false;
    tl_pdl = pdl;
    throw;
  }
  c->prof.suppress = false;
  MGD_CUDA(cudaStreamEndCapture(c->s_body, &recorded));
  launch_inner_end<T>(d, nd, st.maxn, c->s);  // after the conditional node: a plain edge
  tl_pdl = pdl;
}

template <typename T>
static void run_invert(mgd_ctx* c, const Step& st, bool trans) {
  std::vector<int> jac, vc;
  for (int id : st.ops) (c->ops[id].jacobi ? jac : vc).push_back(id);
  apply_jacobi_ops<T>(c, jac, trans);
  if (vc.empty()) return;
  auto& B = batches<T>(c)[st.batch];
  if (!trans && st.loop) {
    run_inner_loop<T>(c, st, B);
    return;
  }
  int maxcount = 1;
  for (int id : vc) maxcount = std::max(maxcount, c->ops[id].count);
  if (maxcount == 1) {
    run_vbatch<T>(B, trans, c->s, c->prof);
    return;
  }
  // several V-cycles: x = V b; repeat: x += V (b - A x)   (per operator)
  for (int id : vc) {
    InvOp& op = c->ops[id];
    MGD_CUDA(cudaMemcpyAsync(op.bsave, op.b, sizeof(T) * op.n, cudaMemcpyDeviceToDevice, c->s));
  }
  run_vbatch<T>(B, trans, c->s, c->prof);
  for (int id : vc) {
    InvOp& op = c->ops[id];
    MGD_CUDA(cudaMemcpyAsync(op.xacc, op.x, sizeof(T) * op.n, cudaMemcpyDeviceToDevice, c->s));
  }
  for (int k = 1; k < maxcount; ++k) {
    for (int id : vc) {
      InvOp& op = c->ops[id];
      Level& l0 = op.h.L[0];
      const Csr& A = trans ? l0.AT : l0.A;
      const T* av = pick<T>(A.v, trans ? l0.atv32 : l0.v32);
      if (k < op.count)
        launch_residual<T>(FMT_CSR4, op.n, A.rp, A.ci, av, nullptr, nullptr, nullptr, (const T*)op.bsave,
                           (const T*)op.xacc, (T*)op.b, c->s);
      else
        MGD_CUDA(cudaMemsetAsync(op.b, 0, sizeof(T) * op.n, c->s));
    }
    run_vbatch<T>(B, trans, c->s, c->prof);
    for (int id : vc) {
      InvOp& op = c->ops[id];
      if (k < op.count) launch_axpy<T>(op.n, (T*)op.xacc, (const T*)op.x, c->s);
    }
  }
  for (int id : vc) {
    InvOp& op = c->ops[id];
    MGD_CUDA(cudaMemcpyAsync(op.x, op.xacc, sizeof(T) * op.n, cudaMemcpyDeviceToDevice, c->s));
    MGD_CUDA(cudaMemcpyAsync(op.b, op.bsave, sizeof(T) * op.n, cudaMemcpyDeviceToDevice, c->s));
  }
}

template <typename T>
static void run_step(mgd_ctx* c, const Step& st, bool trans) {
  {
    switch (st.type) {
      case Step::PRODUCE: {
        int id = c->prof.begin(c->s, 4);
        launch_produce<T>((const ProduceDesc<T>*)st.descs, st.nd, st.len, c->io, c->s);
        c->prof.end(id, 4, st.bytes, c->s);
        break;
      }
      case Step::CONSUME: {
        int id = c->prof.begin(c->s, 4);
        launch_consume<T>((const ConsumeDesc<T>*)st.descs, st.nd, st.len, c->io, c->s);
        c->prof.end(id, 4, st.bytes, c->s);
        break;
      }
      case Step::CONSPROD: {
        int id = c->prof.begin(c->s, 4);
        launch_consume_produce<T>((const ConsumeDesc<T>*)st.descs, st.nd, (const ProduceDesc<T>*)st.descs2, st.nd2,
                                  st.len, c->io, c->s);
        c->prof.end(id, 4, st.bytes, c->s);
        break;
      }
      case Step::INVERT:
        run_invert<T>(c, st, trans);
        break;
      case Step::BLOCKRESID: {
        int id = c->prof.begin(c->s, 4);
        launch_block_resid(c->N, c->bd.nc, (const int* const*)c->bd.d_brp, (const int* const*)c->bd.d_bci,
                           (const double* const*)c->bd.d_bv, (const double* const*)c->bd.d_dtab, c->io,
                           c->rfull, c->s);
        c->prof.end(id, 4, st.bytes, c->s);
        break;
      }
    }
  }
}

// Build the step program of each preconditioner kind and group the inverse
// operators of each INVERT step into V-cycle batches.
template <typename T>
static void build_program(mgd_ctx* c) {
  const int G = c->G, N = c->N, nc = G + 2, E = G, I = G + 1;
  BlockData& bd = c->bd;
  auto D = [&](int a, int b) -> const double* { return bd.d.empty() ? nullptr : bd.d[a * nc + b]; };
  std::vector<Step>& S = c->steps;
  S.clear();
  auto blk = [&](int a) { return (long long)a * N; };
  std::vector<int> opA(nc, -1);
  auto produce1 = [&](int op, PRef a, std::vector<std::tuple<const double*, PRef, double>> t) {
    std::vector<ProduceDesc<T>> v;
    add_produce<T>(c, v, op, a, t);
    push_produce<T>(c, S, v, c->ops[op].n);
  };
  auto consume1 = [&](int op, PRef dst, PRef base, double s) {
    std::vector<ConsumeDesc<T>> v;
    add_consume<T>(v, dst, base, s, c->ops[op].x);
    push_consume<T>(c, S, v, c->ops[op].n);
  };
  switch (c->kind) {
    case MGD_AMG: {
      int op = 0;
      produce1(op, VIN(0), {});
      push_invert(S, {op});
      consume1(op, ZOUT(0), NUL(), 1.0);
      break;
    }
    case MGD_BD: {
      std::vector<ProduceDesc<T>> pv;
      std::vector<ConsumeDesc<T>> cv;
      std::vector<int> all;
      for (int a = 0; a < nc; ++a) {
        add_produce<T>(c, pv, a, VIN(blk(a)), {});
        add_consume<T>(cv, ZOUT(blk(a)), NUL(), 1.0, c->ops[a].x);
        all.push_back(a);
      }
      push_produce<T>(c, S, pv, N);
      push_invert(S, all);
      push_consume<T>(c, S, cv, N);
      break;
    }
    case MGD_BLT: {
      std::vector<ProduceDesc<T>> pv;
      std::vector<ConsumeDesc<T>> cv;
      std::vector<int> groups;
      for (int g = 0; g < G; ++g) {
        add_produce<T>(c, pv, g, VIN(blk(g)), {});
        add_consume<T>(cv, ZOUT(blk(g)), NUL(), 1.0, c->ops[g].x);
        groups.push_back(g);
      }
      push_produce<T>(c, S, pv, N);
      push_invert(S, groups);
      push_consume<T>(c, S, cv, N);
      std::vector<std::tuple<const double*, PRef, double>> t;
      for (int g = 0; g < G; ++g)
        if (D(E, g)) t.emplace_back(D(E, g), ZOUT(blk(g)), -1.0);
      produce1(E, VIN(blk(E)), t);
      push_invert(S, {E});
      consume1(E, ZOUT(blk(E)), NUL(), 1.0);
      t.clear();
      if (D(I, E)) t.emplace_back(D(I, E), ZOUT(blk(E)), -1.0);
      produce1(I, VIN(blk(I)), t);
      push_invert(S, {I});
      consume1(I, ZOUT(blk(I)), NUL(), 1.0);
      break;
    }
    case MGD_SCHUR1: {
      // ops: 0 = A_I, 1 = C_E (option #4: A_E), 2.. = C_g
      int oAI = 0, oCE = 1;
      const int K4 = c->o.opt4_steps;
      std::vector<std::tuple<const double*, PRef, double>> t;
      // option #4 for C_E = A_E - D_EI A_I^-1 D_IE: q = base + sum(qterms); the
      // first step is w = A_E^-1 q, each further one t = A_I^-1 (D_IE w),
      // w = A_E^-1 (q + D_EI t); the last result goes to (dst, dbase, ds)
      auto opt4_CE = [&](PRef qbase, std::vector<std::tuple<const double*, PRef, double>> qterms, PRef dst,
                         PRef dbase, double ds) {
        produce1(oCE, qbase, qterms);
        push_invert(S, {oCE});
        for (int k = 1; k < K4; ++k) {
          consume1(oCE, ABS(c->t4a), NUL(), 1.0);                           // w(k)
          std::vector<std::tuple<const double*, PRef, double>> ti;
          if (D(I, E)) ti.emplace_back(D(I, E), ABS(c->t4a), 1.0);
          produce1(oAI, NUL(), ti);
          push_invert(S, {oAI});
          consume1(oAI, ABS(c->t4b), NUL(), 1.0);                           // A_I^-1 D_IE w(k)
          auto qt = qterms;
          if (D(E, I)) qt.emplace_back(D(E, I), ABS(c->t4b), 1.0);
          produce1(oCE, qbase, qt);
          push_invert(S, {oCE});
        }
        consume1(oCE, dst, dbase, ds);
      };
      produce1(oAI, VIN(blk(I)), {});                                       // 1
      push_invert(S, {oAI});
      consume1(oAI, ABS(c->wIs), NUL(), 1.0);
      if (D(E, I)) t.emplace_back(D(E, I), ABS(c->wIs), -1.0);               // 2
      if (K4 > 0) {
        opt4_CE(VIN(blk(E)), t, ABS(c->wEs), NUL(), 1.0);
      } else {
        produce1(oCE, VIN(blk(E)), t);
        push_invert(S, {oCE});
        consume1(oCE, ABS(c->wEs), NUL(), 1.0);
      }
      std::vector<ProduceDesc<T>> pv;                                        // 3
      std::vector<ConsumeDesc<T>> cv;
      std::vector<int> gs;
      for (int g = 0; g < G; ++g) {
        t.clear();
        if (D(g, E)) t.emplace_back(D(g, E), ABS(c->wEs), -1.0);
        add_produce<T>(c, pv, 2 + g, VIN(blk(g)), t);
        add_consume<T>(cv, ZOUT(blk(g)), NUL(), 1.0, c->ops[2 + g].x);
        gs.push_back(2 + g);
      }
      push_produce<T>(c, S, pv, N);
      push_invert(S, gs);
      push_consume<T>(c, S, cv, N);
      t.clear();                                                             // 4
      for (int g = 0; g < G; ++g)
        if (D(E, g)) t.emplace_back(D(E, g), ZOUT(blk(g)), 1.0);
      if (K4 > 0) {
        opt4_CE(NUL(), t, ZOUT(blk(E)), ABS(c->wEs), -1.0);
      } else {
        produce1(oCE, NUL(), t);
        push_invert(S, {oCE});
        consume1(oCE, ZOUT(blk(E)), ABS(c->wEs), -1.0);
      }
      t.clear();                                                             // 5
      if (D(I, E)) t.emplace_back(D(I, E), ZOUT(blk(E)), 1.0);
      produce1(oAI, NUL(), t);
      push_invert(S, {oAI});
      consume1(oAI, ZOUT(blk(I)), ABS(c->wIs), -1.0);
      break;
    }
    case MGD_SCHUR2: {
      // ops: 0 = A_E, 1..G = S_g, G+1 = S_I
      int oAE = 0, oSI = G + 1;
      std::vector<std::tuple<const double*, PRef, double>> t;
      produce1(oAE, VIN(blk(E)), {});                                        // 1
      push_invert(S, {oAE});
      consume1(oAE, ABS(c->wEs), NUL(), 1.0);
      std::vector<ProduceDesc<T>> pv;                                        // 2
      std::vector<ConsumeDesc<T>> cv;
      std::vector<int> gs;
      for (int g = 0; g < G; ++g) {
        t.clear();
        if (D(g, E)) t.emplace_back(D(g, E), ABS(c->wEs), -1.0);
        add_produce<T>(c, pv, 1 + g, VIN(blk(g)), t);
        add_consume<T>(cv, ZOUT(blk(g)), NUL(), 1.0, c->ops[1 + g].x);
        gs.push_back(1 + g);
      }
      t.clear();
      if (D(I, E)) t.emplace_back(D(I, E), ABS(c->wEs), -1.0);
      add_produce<T>(c, pv, oSI, VIN(blk(I)), t);
      add_consume<T>(cv, ZOUT(blk(I)), NUL(), 1.0, c->ops[oSI].x);
      gs.push_back(oSI);
      push_produce<T>(c, S, pv, N);
      push_invert(S, gs);
      push_consume<T>(c, S, cv, N);
      // option #4 for S_I = A_I - D_IE A_E^-1 D_EI: the step above is w(1) =
      // A_I^-1 q (op G+1 holds A_I); each further step t = A_E^-1 (D_EI w(k)),
      // w(k+1) = A_I^-1 (q + D_IE t), with q = b_I - D_IE w_E* rebuilt from v
      for (int k = 1; k < c->o.opt4_steps; ++k) {
        std::vector<std::tuple<const double*, PRef, double>> te;
        if (D(E, I)) te.emplace_back(D(E, I), ZOUT(blk(I)), 1.0);
        produce1(oAE, NUL(), te);
        push_invert(S, {oAE});
        consume1(oAE, ABS(c->t4a), NUL(), 1.0);
        auto qt = t;
        if (D(I, E)) qt.emplace_back(D(I, E), ABS(c->t4a), 1.0);
        produce1(oSI, VIN(blk(I)), qt);
        push_invert(S, {oSI});
        consume1(oSI, ZOUT(blk(I)), NUL(), 1.0);
      }
      t.clear();                                                             // 3
      for (int g = 0; g < G; ++g)
        if (D(E, g)) t.emplace_back(D(E, g), ZOUT(blk(g)), 1.0);
      if (D(E, I)) t.emplace_back(D(E, I), ZOUT(blk(I)), 1.0);
      produce1(oAE, NUL(), t);
      push_invert(S, {oAE});
      consume1(oAE, ZOUT(blk(E)), ABS(c->wEs), -1.0);
      break;
    }
    case MGD_PCTL: {
      // ops: 0..nc-1 = A_a, nc = A_c
      int oAc = nc;
      produce1(E, VIN(blk(E)), {});                                          // 1: E first
      push_invert(S, {E});
      consume1(E, ZOUT(blk(E)), NUL(), 1.0);
      std::vector<ProduceDesc<T>> pv;
      std::vector<ConsumeDesc<T>> cv;
      std::vector<int> others;
      for (int a = 0; a < nc; ++a) {
        if (a == E) continue;
        std::vector<std::tuple<const double*, PRef, double>> t;
        if (D(a, E)) t.emplace_back(D(a, E), ZOUT(blk(E)), -1.0);
        add_produce<T>(c, pv, a, VIN(blk(a)), t);
        add_consume<T>(cv, ZOUT(blk(a)), NUL(), 1.0, c->ops[a].x);
        others.push_back(a);
      }
      push_produce<T>(c, S, pv, N);
      push_invert(S, others);
      push_consume<T>(c, S, cv, N);
      Step br;                                                               // 2: r = b - A w
      br.type = Step::BLOCKRESID;
      br.bytes = 0;
      for (int a = 0; a < nc; ++a) br.bytes += sp_bytes(bd.Ab[a].nnz, N, 8) + 24.0 * N;
      S.push_back(br);
      std::vector<std::tuple<const double*, PRef, double>> t;
      for (int a = 0; a < nc; ++a) t.emplace_back(a == E ? nullptr : bd.p[a], ABS(c->rfull + blk(a)), 1.0);
      produce1(oAc, NUL(), t);
      push_invert(S, {oAc});
      // 3: w_a += p_a (.) w_c with p_E = 1: w_c to FP64, then a z-relative update
      std::vector<ConsumeDesc<T>> cc;
      add_consume<T>(cc, ABS(c->wEs), NUL(), 1.0, c->ops[oAc].x);  // w_c in FP64
      push_consume<T>(c, S, cc, N);
      Step upd;
      upd.type = Step::PRODUCE;
      {
        // destination offsets relative to the z slot (dst holds the offset)
        std::vector<ProduceDesc<double>> zp;
        for (int a = 0; a < nc; ++a) {
          ProduceDesc<double> d;
          memset(&d, 0, sizeof(d));
          d.dst = reinterpret_cast<double*>((long long)blk(a));  // offset, resolved against z
          d.a = ZOUT(blk(a));
          d.nt = 1;
          d.d[0] = a == E ? nullptr : bd.p[a];
          d.w[0] = ABS(c->wEs);
          d.s[0] = 1.0;
          zp.push_back(d);
        }
        upd.descs = upload_vec(c, zp);
        upd.nd = nc;
        upd.len = N;
        upd.bytes = nc * 32.0 * N;
        upd.batch = -2;  // marks the z-relative FP64 update
      }
      S.push_back(upd);
      break;
    }
  }
  // a CONSUME and the PRODUCE right after it run as one elementwise kernel
  std::vector<Step> fused;
  for (size_t i = 0; i < S.size(); ++i) {
    if (i + 1 < S.size() && S[i].type == Step::CONSUME && S[i + 1].type == Step::PRODUCE && S[i].batch == -1 &&
        S[i + 1].batch == -1 && S[i].len == S[i + 1].len && S[i].nd <= kCpMaxCons && S[i + 1].nd <= kCpMaxProd &&
        S[i + 1].nterms <= kCpMaxTerms) {
      Step f = S[i];
      f.type = Step::CONSPROD;
      f.descs2 = S[i + 1].descs;
      f.nd2 = S[i + 1].nd;
      f.bytes = S[i].bytes + S[i + 1].bytes;
      fused.push_back(f);
      ++i;
      continue;
    }
    fused.push_back(S[i]);
  }
  S = fused;
}

}  // namespace mgd

// z-relative FP64 update kernel used by the PCTL coarse-grid correction
namespace mgd {
__global__ void k_zupdate(const ProduceDesc<double>* __restrict__ ds, int N, const IOSlots* __restrict__ io) {
  const ProduceDesc<double>* d = ds + blockIdx.y;
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  double* z = io->z + (long long)d->dst;
  const double* w = d->w[0].abs;
  double t = w[k];
  if (d->d[0]) t *= d->d[0][k];
  z[k] = z[k] + t;
}
}  // namespace mgd

namespace mgd {

template <typename T>
static void run_program(mgd_ctx* c, bool trans) {
  for (const Step& st : c->steps) {
    if (st.type == Step::PRODUCE && st.batch == -2) {
      int id = c->prof.begin(c->s, 4);
      k_zupdate<<<dim3(cdiv(st.len, kThreads), st.nd), kThreads, 0, c->s>>>(
          (const ProduceDesc<double>*)st.descs, st.len, c->io);
      MGD_LAUNCH_CHECK();
      c->prof.end(id, 4, st.bytes, c->s);
      continue;
    }
    run_step<T>(c, st, trans);
  }
}

// Autotuner decisions keyed by the batch's shape (value type, depth, and per
// level the subsystem count, largest row count and nonzeros): a setup of a
// system with the same hierarchy shape reuses them instead of re-timing.
struct TuneResult {
  std::vector<int> fmtA, fmtR, fmtP, fmtGS;
  int tail_level;
  int tail_cs = 8;
};
static std::mutex g_tune_mu;
static std::map<std::vector<long long>, TuneResult> g_tune_cache;

// With the environment variable MGD_TUNE_CACHE naming a file, the decisions
// also persist across processes: the file is read at the first lookup and
// rewritten (through a per-process temporary file and a rename) after every
// new decision.  One line per entry, fields separated by '|': the key, fmtA,
// fmtR, fmtP, fmtGS, then tail_level and tail_cs.  Lines that do not parse
// are skipped.  Callers hold g_tune_mu.
static bool g_tune_loaded = false;

static const char* tune_file() {
  const char* p = std::getenv("MGD_TUNE_CACHE");
  return p && *p ? p : nullptr;
}

template <typename V>
static bool parse_ints(const std::string& f, std::vector<V>& out) {
  std::istringstream is(f);
  long long x;
  out.clear();
  while (is >> x) out.push_back((V)x);
  return is.eof();
}

static void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = tune_file();
  if (!path) return;
  std::ifstream in(path);
  std::string line;
  while (std::getline(in, line)) {
    std::vector<std::string> f;
    std::string cur;
    for (char ch : line) {
      if (ch == '|') {
        f.push_back(cur);
        cur.clear();
      } else {
        cur.push_back(ch);
      }
    }
    f.push_back(cur);
    if (f.size() != 6) continue;
    std::vector<long long> key;
    TuneResult r;
    std::vector<int> tail;
    if (!parse_ints(f[0], key) || key.empty() || !parse_ints(f[1], r.fmtA) || !parse_ints(f[2], r.fmtR) ||
        !parse_ints(f[3], r.fmtP) || !parse_ints(f[4], r.fmtGS) || !parse_ints(f[5], tail) || tail.size() != 2)
      continue;
    r.tail_level = tail[0];
    r.tail_cs = tail[1];
    g_tune_cache[key] = r;
  }
}

static void tune_save_locked() {
  const char* path = tune_file();
  if (!path) return;
  std::string tmp = std::string(path) + ".tmp." + std::to_string((long long)getpid());
  {
    std::ofstream out(tmp, std::ios::trunc);
    if (!out) return;
    auto put = [&](const auto& v) {
      for (size_t i = 0; i < v.size(); ++i) out << (i ? " " : "") << v[i];
    };
    for (const auto& kv : g_tune_cache) {
      put(kv.first);
      out << '|';
      put(kv.second.fmtA);
      out << '|';
      put(kv.second.fmtR);
      out << '|';
      put(kv.second.fmtP);
      out << '|';
      put(kv.second.fmtGS);
      out << '|' << kv.second.tail_level << ' ' << kv.second.tail_cs << '\n';
    }
    if (!out) return;
  }
  std::rename(tmp.c_str(), path);
}

template <typename T>
static std::vector<long long> tune_key(const VBatch<T>& vb, bool trans, int fuse_rows, bool graph) {
  std::vector<long long> k{(long long)sizeof(T), vb.depth, trans ? 1 : 0, fuse_rows, graph ? 1 : 0};
  for (int l = 0; l < vb.depth; ++l) {
    long long nnz = 0;
    for (Hier* h : vb.hs)
      if (l < h->nlev()) nnz += h->L[l].A.nnz;
    k.push_back(vb.plan[l].gs ? vb.plan[l].nkmax : -1);
    k.push_back(vb.plan[l].ndown);
    k.push_back(vb.plan[l].maxn);
    k.push_back(nnz);
  }
  return k;
}

// group INVERT steps into batches (one batch per step when batched, else one per op)
// INVERT steps whose V-cycle operators need the device-controlled loop
// (option #3, or more than one cycle): a flag per hierarchy (read by the
// V-cycle kernels, so it must exist before the plans are built), the loop
// descriptors and the loop state.
template <typename T>
static void setup_loops(mgd_ctx* c) {
  static const int kOne = 1;
  for (Step& st : c->steps) {
    if (st.type != Step::INVERT || st.batch < 0) continue;
    std::vector<int> vc;
    bool need = false;
    for (int id : st.ops) {
      const InvOp& op = c->ops[id];
      if (op.jacobi) continue;
      vc.push_back(id);
      need = need || op.accurate || op.count > 1;
    }
    if (!need) continue;
    std::vector<InnerDesc<T>> ds;
    int maxn = 0, guard = std::max(1, c->o.inner_maxit);
    for (int id : vc) {
      InvOp& op = c->ops[id];
      const size_t es = sizeof(T);
      if (!op.h.active) {
        op.h.active = c->ar.alloc<int>(1);
        MGD_CUDA(cudaMemcpyAsync(op.h.active, &kOne, sizeof(int), cudaMemcpyHostToDevice, c->s));
      }
      if (!op.bsave) op.bsave = c->ar.alloc<char>(es * op.n, true, c->s);
      if (!op.xacc) op.xacc = c->ar.alloc<char>(es * op.n, true, c->s);
      Level& l0 = op.h.L[0];
      InnerDesc<T> d;
      memset(&d, 0, sizeof(d));
      d.rp = l0.A.rp;
      d.ci = l0.A.ci;
      d.v = pick<T>(l0.A.v, l0.v32);
      d.b = (T*)op.b;
      d.x = (T*)op.x;
      d.rhs = (T*)op.bsave;
      d.xacc = (T*)op.xacc;
      d.n = op.n;
      d.accurate = op.accurate ? 1 : 0;
      d.count = op.count;
      d.active = op.h.active;
      ds.push_back(d);
      maxn = std::max(maxn, op.n);
      guard = std::max(guard, op.count);
    }
    const int nd = (int)ds.size();
    InnerCtl h;
    memset(&h, 0, sizeof(h));
    h.nops = nd;
    h.maxit = std::max(1, c->o.inner_maxit);
    h.guard = guard;
    h.tol = c->o.inner_tol;
    h.part = c->ar.alloc<double>((size_t)nd * kInnerParts, true, c->s);
    h.nr0 = c->ar.alloc<double>(nd, true, c->s);
    h.cycles = c->ar.alloc<int>(nd, true, c->s);
    h.total = c->ar.alloc<long long>(nd, true, c->s);
    h.trips = c->ar.alloc<int>(1, true, c->s);
    h.any = c->ar.alloc<int>(1, true, c->s);
    st.loop = true;
    st.loop_ops = vc;
    st.maxn = maxn;
    st.guard = guard;
    st.total = h.total;
    st.any = h.any;
    st.inner = upload_vec(c, ds);
    st.ctl = (InnerCtl*)upload_vec(c, std::vector<InnerCtl>{h});
  }
}

template <typename T>
static void build_batches(mgd_ctx* c) {
  auto& B = batches<T>(c);
  B.clear();
  std::vector<Step> out;
  for (Step& st : c->steps) {
    if (st.type != Step::INVERT) {
      out.push_back(st);
      continue;
    }
    std::vector<int> vc;
    for (int id : st.ops)
      if (!c->ops[id].jacobi) vc.push_back(id);
    std::vector<int> jac;
    for (int id : st.ops)
      if (c->ops[id].jacobi) jac.push_back(id);
    if (c->o.batched || vc.size() <= 1) {
      Step s2 = st;
      if (!vc.empty()) {
        B.emplace_back();
        for (int id : vc) B.back().hs.push_back(&c->ops[id].h);
        s2.batch = (int)B.size() - 1;
      }
      out.push_back(s2);
    } else {
      // one step per operator (plain launches)
      bool first = true;
      for (int id : vc) {
        Step s2 = st;
        s2.ops = {id};
        if (first) {
          for (int j : jac) s2.ops.push_back(j);
          first = false;
        }
        B.emplace_back();
        B.back().hs.push_back(&c->ops[id].h);
        s2.batch = (int)B.size() - 1;
        out.push_back(s2);
      }
    }
  }
  c->steps = out;
  setup_loops<T>(c);
  for (auto& vb : B) {
    build_plan<T>(c->ar, vb, false, c->s);
    if (c->o.keep_transpose) build_plan<T>(c->ar, vb, true, c->s);
    bool cached = false;
    std::vector<long long> key = tune_key<T>(vb, false, c->o.fuse_rows, c->o.use_graph != 0 && c->s != nullptr);
    if (c->o.autotune) {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      tune_load_locked();
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end() && (int)it->second.fmtA.size() == vb.depth) {
        for (int l = 0; l < vb.depth; ++l) {
          vb.plan[l].fmtA = it->second.fmtA[l];
          vb.plan[l].fmtR = it->second.fmtR[l];
          vb.plan[l].fmtP = it->second.fmtP[l];
          vb.plan[l].fmtGS = it->second.fmtGS[l];
          if (c->o.keep_transpose) {
            vb.planT[l].fmtA = it->second.fmtA[l];
            vb.planT[l].fmtR = it->second.fmtR[l];
            vb.planT[l].fmtP = it->second.fmtP[l];
            int f = it->second.fmtGS[l];  // the transposed plan has no sweep-ordered copy
            vb.planT[l].fmtGS = f == FMT_SELL ? FMT_CSR4 : f;
          }
        }
        cached = true;
      }
    }
    if (cached) {
      vb.tail_cs = g_tune_cache[key].tail_cs;
      build_tail<T>(c->ar, vb, g_tune_cache[key].tail_level, c->o.keep_transpose != 0, c->s);
      continue;
    }
    if (c->o.autotune) {
      autotune<T>(vb, false, c->s);
      if (c->o.keep_transpose) autotune<T>(vb, true, c->s);
    }
    if (c->o.fuse_rows > 0) {
      int Lt = vb.depth;
      for (int l = 1; l < vb.depth; ++l) {
        auto& lp = vb.plan[l];
        if (std::max(lp.maxn, std::max(lp.maxcn, lp.maxcj)) <= c->o.fuse_rows) {
          Lt = l;
          break;
        }
      }
      build_tail<T>(c->ar, vb, Lt, c->o.keep_transpose != 0, c->s);
    } else if (c->o.fuse_rows == 0 && c->o.autotune) {
      autotune_tail<T>(c->ar, vb, c->o.keep_transpose != 0, c->o.use_graph != 0 && c->s != nullptr, c->s);
    }
    if (c->o.autotune) {
      TuneResult r;
      for (int l = 0; l < vb.depth; ++l) {
        r.fmtA.push_back(vb.plan[l].fmtA);
        r.fmtR.push_back(vb.plan[l].fmtR);
        r.fmtP.push_back(vb.plan[l].fmtP);
        r.fmtGS.push_back(vb.plan[l].fmtGS);
      }
      r.tail_level = vb.tail_level;
      r.tail_cs = vb.tail_cs;
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune_cache[key] = r;
      tune_save_locked();
    }
  }
}

}  // namespace mgd

using namespace mgd;

// ------------------------------------------------------------------ helpers of the API
static int fail(mgd_ctx* c, const Error& e) {
  if (c) c->err = e.msg;
  return e.code;
}

template <typename F>
static int guarded(mgd_ctx* c, F&& f) {
  if (!c) return MGD_EINVAL;
  try {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != c->device) MGD_CUDA(cudaSetDevice(c->device));
    tl_pool = c->ar.pool;
    tl_stream = nullptr;
    tl_pdl = c->o.pdl != 0;
    int r = f();
    if (dev != c->device) cudaSetDevice(dev);
    return r;
  } catch (const Error& e) {
    return fail(c, e);
  } catch (const std::exception& e) {
    return fail(c, Error{MGD_ECUDA, e.what()});
  }
}

static void precond_apply(mgd_ctx* c, const double* v, double* z, bool trans) {
  (trans ? c->napplyT : c->napply)++;
  launch_set_io(c->io, v, z, c->s);
  if (!trans && c->graph_ok) {
    MGD_CUDA(cudaGraphLaunch(c->graph, c->s));
    __atomic_add_fetch(&g_kernel_launches, c->graph_kernels, __ATOMIC_RELAXED);
    c->prof.graph_replayed = true;
    return;
  }
  if (mixed(c)) run_program<float>(c, trans);
  else run_program<double>(c, trans);
}

static void capture_graph(mgd_ctx* c) {
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  c->graph_ok = false;
  if (!c->o.use_graph) return;
  cudaGraph_t g;
  c->prof.drop_graph_pairs();
  long long k0 = __atomic_load_n(&g_kernel_launches, __ATOMIC_RELAXED);
  c->prof.capturing = true;
  c->capturing = true;
  if (!c->s_body) MGD_CUDA(cudaStreamCreateWithFlags(&c->s_body, cudaStreamNonBlocking));
  MGD_CUDA(cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal));
  try {
    if (mixed(c)) run_program<float>(c, false);
    else run_program<double>(c, false);
  } catch (...) {
    cudaStreamEndCapture(c->s, &g);
    c->prof.capturing = false;
    c->capturing = false;
    throw;
  }
  c->prof.capturing = false;
  c->capturing = false;
  MGD_CUDA(cudaStreamEndCapture(c->s, &g));
  // kernels recorded into the graph (the counter counted them at capture)
  long long k1 = __atomic_load_n(&g_kernel_launches, __ATOMIC_RELAXED);
  c->graph_kernels = k1 - k0;
  __atomic_sub_fetch(&g_kernel_launches, c->graph_kernels, __ATOMIC_RELAXED);
  MGD_CUDA(cudaGraphInstantiate(&c->graph, g, 0));
  cudaGraphDestroy(g);
  c->graph_ok = true;
}

static void free_setup(mgd_ctx* c) {
  if (c->s) cudaStreamSynchronize(c->s);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  c->graph = nullptr;
  c->graph_ok = false;
  c->ar.release();
  c->ops.clear();
  c->steps.clear();
  c->vb64.clear();
  c->vb32.clear();
  c->bd = BlockData();
  c->ready = false;
  c->napply = c->napplyT = 0;
}

// free_setup, timed (ms): do_setup resets the phase clock, so callers record it afterwards
static double free_setup_timed(mgd_ctx* c) {
  const auto t = std::chrono::steady_clock::now();
  free_setup(c);
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t).count();
}

static void record_phase(mgd_ctx* c, int ph, double ms) {
  std::lock_guard<std::mutex> lk(c->phases.mu);
  c->phases.ms[ph] = ms;
}

// owned: rp, ci, v are arrays of the context's arena (mgd_setup_host copied
// the host arrays there), kept as the monolithic operator without a copy
static void do_setup(mgd_ctx* c, const int* rp, const int* ci, const double* v, bool owned = false) {
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = c->s;
  int G = c->G, N = c->N, n = c->n, nnz = c->nnz, nc = G + 2;
  const mgd_opts& o = c->o;
  c->ar.stream = s;
  c->phases.reset();
  PhaseTimer pt_val(&c->phases, SP_VALIDATE);
  // validation
  {
    Scratch sc(s);
    int* flags = sc.alloc<int>(5);
    MGD_CUDA(cudaMemsetAsync(flags, 0, 5 * sizeof(int), s));
    launch_validate(n, nnz, N, nc, rp, ci, v, flags, s);
    int hf[5];
    MGD_CUDA(cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, s));
    MGD_CUDA(cudaStreamSynchronize(s));
    if (hf[3]) throw Error{MGD_EINVAL, "row pointer does not span [0, nnz]"};
    if (hf[0]) throw Error{MGD_EINVAL, "column index out of range, unsorted or duplicated"};
    if (hf[1]) throw Error{MGD_EINVAL, "off-block entry couples different cells (D_ab must be diagonal)"};
    if (hf[4]) throw Error{MGD_ENAN, "a matrix value is not finite"};
    if (hf[2]) throw Error{MGD_EINVAL, "missing or non-positive diagonal entry"};
  }
  // keep a copy of the monolithic operator
  Csr in;
  in.n = n;
  in.m = n;
  in.nnz = nnz;
  in.rp = const_cast<int*>(rp);
  in.ci = const_cast<int*>(ci);
  in.v = const_cast<double*>(v);
  c->A = owned ? in : csr_copy(c->ar, in, s);
  c->Asell = build_sell(c->ar, c->A, false, s);
  if (o.keep_transpose) {
    c->AT = transpose(c->ar, c->A, s);
    c->ATsell = build_sell(c->ar, c->AT, false, s);
  }
  pt_val.stop();
  PhaseTimer pt_blk(&c->phases, SP_BLOCKS);
  c->wEs = c->ar.alloc<double>(N, true);
  c->wIs = c->ar.alloc<double>(N, true);
  c->t4a = c->ar.alloc<double>(N, true);
  c->t4b = c->ar.alloc<double>(N, true);
  c->rfull = c->ar.alloc<double>(n, true);
  c->io = c->ar.alloc<IOSlots>(1, true);
  c->ops.clear();
  c->n_jacobi = 0;
  int ndrop = 0;
  if (c->kind == MGD_AMG) {
    add_op(c, OP_MONO, 0, c->A);
  } else {
    // block extraction
    BlockData& bd = c->bd;
    bd.G = G;
    bd.N = N;
    bd.nc = nc;
    Scratch sc(s);
    int* cnt = sc.alloc<int>(n);
    int* pairs = sc.alloc<int>(nc * nc);
    MGD_CUDA(cudaMemsetAsync(pairs, 0, sizeof(int) * nc * nc, s));
    launch_block_count(n, N, nc, c->A.rp, c->A.ci, cnt, pairs, s);
    int* brp = sc.alloc<int>(n + 1);
    exclusive_scan(cnt, brp, n, s);
    int tot = read_int(brp + n, s);
    std::vector<int> hpairs(nc * nc);
    MGD_CUDA(cudaMemcpyAsync(hpairs.data(), pairs, sizeof(int) * nc * nc, cudaMemcpyDeviceToHost, s));
    MGD_CUDA(cudaStreamSynchronize(s));
    bd.d.assign(nc * nc, nullptr);
    bd.dropped.assign(nc * nc, 0);
    for (int k = 0; k < nc * nc; ++k)
      if (hpairs[k]) bd.d[k] = c->ar.alloc<double>(N, true);
    double** dtab = sc.alloc<double*>(nc * nc);
    MGD_CUDA(cudaMemcpyAsync(dtab, bd.d.data(), sizeof(double*) * nc * nc, cudaMemcpyHostToDevice, s));
    int* bci = c->ar.alloc<int>(tot);
    double* bv = c->ar.alloc<double>(tot);
    launch_block_fill(n, N, nc, c->A.rp, c->A.ci, c->A.v, brp, bci, bv, dtab, s);
    // each block's row pointer is made on the device; only the nc + 1 block
    // boundaries come back to the host
    std::vector<int*> hrps(nc);
    for (int a = 0; a < nc; ++a) hrps[a] = c->ar.alloc<int>(N + 1);
    int** drps = sc.alloc<int*>(nc);
    MGD_CUDA(cudaMemcpyAsync(drps, hrps.data(), sizeof(int*) * nc, cudaMemcpyHostToDevice, s));
    launch_block_rowptr(N, nc, brp, drps, s);
    int* bounds = sc.alloc<int>(nc + 1);
    launch_block_bounds(N, nc, brp, bounds, s);
    std::vector<int> hb(nc + 1);
    MGD_CUDA(cudaMemcpyAsync(hb.data(), bounds, sizeof(int) * (nc + 1), cudaMemcpyDeviceToHost, s));
    MGD_CUDA(cudaStreamSynchronize(s));
    bd.Ab.resize(nc);
    bd.diag.resize(nc);
    for (int a = 0; a < nc; ++a) {
      Csr B;
      B.n = N;
      B.m = N;
      B.nnz = hb[a + 1] - hb[a];
      B.rp = hrps[a];
      B.ci = bci + hb[a];
      B.v = bv + hb[a];
      bd.Ab[a] = B;
      bd.diag[a] = c->ar.alloc<double>(N);
      launch_diag_extract(N, B.rp, B.ci, B.v, bd.diag[a], s);
    }
    // Section 3.6: drop D_ab when gamma_wc^{ab} > sigma_wc
    if (o.adaptive) {
      int* cntw = sc.alloc<int>(1);
      for (int a = 0; a < nc; ++a)
        for (int b = 0; b < nc; ++b) {
          double* d = bd.d[a * nc + b];
          if (!d) continue;
          MGD_CUDA(cudaMemsetAsync(cntw, 0, sizeof(int), s));
          launch_gamma_wc(N, d, bd.diag[a], o.theta_wc, cntw, s);
          double g = (double)read_int(cntw, s) / N;
          if (g > o.sigma_wc) {
            bd.d[a * nc + b] = nullptr;
            bd.dropped[a * nc + b] = 1;
            ++ndrop;
          }
        }
    }
    auto D = [&](int a, int b) -> const double* { return bd.d[a * nc + b]; };
    int E = G, I = G + 1;
    switch (c->kind) {
      case MGD_BD:
      case MGD_BLT:
        for (int a = 0; a < nc; ++a) add_op(c, OP_A, a, csr_copy(c->ar, bd.Ab[a], s));
        break;
      case MGD_SCHUR1: {
        add_op(c, OP_A, I, csr_copy(c->ar, bd.Ab[I], s));
        Csr CE = diag_modified(c, bd.Ab[E], D(E, I), D(I, E), bd.diag[I]);
        double* dCE = c->ar.alloc<double>(N);
        launch_diag_extract(N, CE.rp, CE.ci, CE.v, dCE, s);
        if (o.opt4_steps > 0)  // option #4: C_E^-1 by the recurrence on A_E and A_I (C_E-hat gives C_g-hat its diagonal)
          add_op(c, OP_A, E, csr_copy(c->ar, bd.Ab[E], s));
        else
          add_op(c, OP_CE, E, CE);
        for (int g = 0; g < G; ++g) add_op(c, OP_CG, g, diag_modified(c, bd.Ab[g], D(g, E), D(E, g), dCE));
        break;
      }
      case MGD_SCHUR2:
        add_op(c, OP_A, E, csr_copy(c->ar, bd.Ab[E], s));
        for (int g = 0; g < G; ++g) add_op(c, OP_SG, g, diag_modified(c, bd.Ab[g], D(g, E), D(E, g), bd.diag[E]));
        if (o.opt4_steps > 0)  // option #4: S_I^-1 by the recurrence on A_I and A_E
          add_op(c, OP_A, I, csr_copy(c->ar, bd.Ab[I], s));
        else
          add_op(c, OP_SI, I, diag_modified(c, bd.Ab[I], D(I, E), D(E, I), bd.diag[E]));
        break;
      case MGD_PCTL:
        for (int a = 0; a < nc; ++a) add_op(c, OP_A, a, csr_copy(c->ar, bd.Ab[a], s));
        break;
    }
    // device tables of the blocks
    std::vector<int*> hrp(nc), hci(nc);
    std::vector<double*> hv(nc);
    for (int a = 0; a < nc; ++a) {
      hrp[a] = bd.Ab[a].rp;
      hci[a] = bd.Ab[a].ci;
      hv[a] = bd.Ab[a].v;
    }
    bd.d_brp = (int**)upload_vec(c, hrp);
    bd.d_bci = (int**)upload_vec(c, hci);
    bd.d_bv = (double**)upload_vec(c, hv);
    bd.d_dtab = (double**)upload_vec(c, bd.d);
  }
  // hierarchies / Jacobi data
  MGD_CUDA(cudaStreamSynchronize(s));
  pt_blk.stop();
  PhaseTimer pt_h(&c->phases, SP_HIERARCHIES);
  if (mixed(c)) finalize_ops_parallel<float>(c, 0, c->ops.size());
  else finalize_ops_parallel<double>(c, 0, c->ops.size());
  pt_h.stop();
  PhaseTimer pt_pctl(&c->phases, SP_PCTL);
  for (auto& op : c->ops)
    if (op.jacobi) c->n_jacobi++;
  if (c->kind == MGD_PCTL) {
    // p_a = -A_a^{-1} D_aE 1 by option #3 (V-cycles until ||r|| <= tol ||rhs||), FP64 arithmetic
    BlockData& bd = c->bd;
    int E = G;
    bd.p.assign(nc, nullptr);
    Scratch sc(s);
    double* rhs = sc.alloc<double>(N);
    double* r = sc.alloc<double>(N);
    double* part = sc.alloc<double>(kDotBlocks * 32);
    double* nrm = sc.alloc<double>(2);
    for (int a = 0; a < nc; ++a) {
      if (a == E) continue;
      bd.p[a] = c->ar.alloc<double>(N, true);
      const double* dE = bd.d[a * nc + E];
      if (!dE) continue;
      launch_lincomb(N, -1.0, dE, 0.0, dE, rhs, s);
      launch_norm2(N, rhs, part, nrm, s);
      double h0;
      MGD_CUDA(cudaMemcpyAsync(&h0, nrm, sizeof(double), cudaMemcpyDeviceToHost, s));
      MGD_CUDA(cudaStreamSynchronize(s));
      double nr0 = std::sqrt(h0);
      InvOp& op = c->ops[a];
      std::vector<Hier*> hh{&op.h};
      VBatch<double> vb64;
      VBatch<float> vb32;
      if (!op.jacobi) {
        if (mixed(c)) {
          vb32.hs = hh;
          build_plan<float>(c->ar, vb32, false, s);
        } else {
          vb64.hs = hh;
          build_plan<double>(c->ar, vb64, false, s);
        }
      }
      for (int it = 0; it < o.inner_maxit; ++it) {
        launch_resid_f64(FMT_CSR4, N, op.A.rp, op.A.ci, op.A.v, nullptr, nullptr, nullptr, rhs, bd.p[a], r, s);
        launch_norm2(N, r, part, nrm, s);
        double h1;
        MGD_CUDA(cudaMemcpyAsync(&h1, nrm, sizeof(double), cudaMemcpyDeviceToHost, s));
        MGD_CUDA(cudaStreamSynchronize(s));
        if (std::sqrt(h1) <= o.inner_tol * nr0) break;
        if (mixed(c)) {
          launch_cast_f64_f32(N, r, (float*)op.b, s);
          if (op.jacobi) {
            JacDesc<float> jd{(float*)op.x, (const float*)op.b, op.jd32};
            JacDesc<float>* dd = sc.alloc<JacDesc<float>>(1);
            MGD_CUDA(cudaMemcpyAsync(dd, &jd, sizeof(jd), cudaMemcpyHostToDevice, s));
            launch_jacobi<float>(dd, 1, N, s);
          } else {
            run_vbatch<float>(vb32, false, s, c->prof);
          }
          Scratch t2(s);
          double* ed = t2.alloc<double>(N);
          launch_cast_f32_f64(N, (const float*)op.x, ed, s);
          launch_saxpy_vec(N, 1.0, ed, bd.p[a], s);
          MGD_CUDA(cudaStreamSynchronize(s));
        } else {
          launch_copy_f64(N, r, (double*)op.b, s);
          if (op.jacobi) {
            JacDesc<double> jd{(double*)op.x, (const double*)op.b, op.jd};
            JacDesc<double>* dd = sc.alloc<JacDesc<double>>(1);
            MGD_CUDA(cudaMemcpyAsync(dd, &jd, sizeof(jd), cudaMemcpyHostToDevice, s));
            launch_jacobi<double>(dd, 1, N, s);
          } else {
            run_vbatch<double>(vb64, false, s, c->prof);
          }
          launch_saxpy_vec(N, 1.0, (const double*)op.x, bd.p[a], s);
        }
      }
    }
    // Eq. 3.3 coarse operator on the union pattern
    int* acnt = sc.alloc<int>(N);
    launch_pctl_ac_count(N, nc, (const int* const*)bd.d_brp, (const int* const*)bd.d_bci, acnt, s);
    Csr Ac;
    Ac.n = N;
    Ac.m = N;
    Ac.rp = c->ar.alloc<int>(N + 1);
    exclusive_scan(acnt, Ac.rp, N, s);
    Ac.nnz = read_int(Ac.rp + N, s);
    Ac.ci = c->ar.alloc<int>(Ac.nnz);
    Ac.v = c->ar.alloc<double>(Ac.nnz);
    std::vector<double*> hp(nc, nullptr);
    for (int a = 0; a < nc; ++a) hp[a] = bd.p[a];
    double** dp = (double**)upload_vec(c, hp);
    launch_pctl_ac_fill(N, nc, G, (const int* const*)bd.d_brp, (const int* const*)bd.d_bci,
                        (const double* const*)bd.d_bv, (const double* const*)dp, (const double* const*)bd.d_dtab,
                        Ac.rp, Ac.ci, Ac.v, s);
    bd.Ac = Ac;
    int oAc = add_op(c, OP_AC, E, Ac);
    if (mixed(c)) finalize_op<float>(c, c->ops[oAc], s);
    else finalize_op<double>(c, c->ops[oAc], s);
    if (c->ops[oAc].jacobi) c->n_jacobi++;
  }
  // program, batches, graph
  pt_pctl.stop();
  PhaseTimer pt_prog(&c->phases, SP_PROGRAM);
  if (mixed(c)) {
    build_program<float>(c);
    build_batches<float>(c);
  } else {
    build_program<double>(c);
    build_batches<double>(c);
  }
  // FGMRES storage
  MGD_CUDA(cudaStreamSynchronize(s));
  pt_prog.stop();
  PhaseTimer pt_kry(&c->phases, SP_KRYLOV);
  c->m = std::max(1, std::min(o.restart, 30));
  c->V = c->ar.alloc<double>((size_t)(c->m + 1) * n, true);
  c->Z = c->ar.alloc<double>((size_t)c->m * n, true);
  c->w = c->ar.alloc<double>(n, true);
  c->r = c->ar.alloc<double>(n, true);
  c->xtmp = c->ar.alloc<double>(n, true);
  c->btmp = c->ar.alloc<double>(n, true);
  c->hbuf = c->ar.alloc<double>(128, true);
  c->partial = c->ar.alloc<double>((size_t)kDotBlocks * 32, true);
  c->ybuf = c->ar.alloc<double>(64, true);
  if (!c->hpin) MGD_CUDA(cudaMallocHost(&c->hpin, 256 * sizeof(double)));  // kept across setups
  c->arn_nb = o.arnoldi_resident ? arnoldi_coop_blocks(n) : 0;
  // monolithic SpMV layout (cached by operator size, like the V-cycle plans)
  c->fmtMono = FMT_SELL;
  const std::vector<long long> mkey{-1, n, c->A.nnz};
  bool mono_cached = false;
  if (o.autotune) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    auto it = g_tune_cache.find(mkey);
    if (it != g_tune_cache.end() && !it->second.fmtA.empty()) {
      c->fmtMono = it->second.fmtA[0];
      mono_cached = true;
    }
  }
  if (o.autotune && !mono_cached) {
    cudaEvent_t e0, e1;
    MGD_CUDA(cudaEventCreate(&e0));
    MGD_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int f : {FMT_SELL, FMT_CSR1, FMT_CSR2, FMT_CSR4, FMT_CSR8}) {
      launch_spmv_f64(f, n, c->A.rp, c->A.ci, c->A.v, c->Asell.sptr, c->Asell.ci, c->Asell.v, c->r, c->w, s);
      MGD_CUDA(cudaEventRecord(e0, s));
      for (int k = 0; k < 6; ++k)
        launch_spmv_f64(f, n, c->A.rp, c->A.ci, c->A.v, c->Asell.sptr, c->Asell.ci, c->Asell.v, c->r, c->w, s);
      MGD_CUDA(cudaEventRecord(e1, s));
      MGD_CUDA(cudaEventSynchronize(e1));
      float ms;
      MGD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        c->fmtMono = f;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    TuneResult r;
    r.fmtA.push_back(c->fmtMono);
    r.tail_level = 0;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[mkey] = r;
    tune_save_locked();
  }
  capture_graph(c);
  MGD_CUDA(cudaStreamSynchronize(s));
  pt_kry.stop();
  // stats
  memset(&c->st, 0, sizeof(c->st));
  mgd_stats& st = c->st;
  st.kind = c->kind;
  st.G = G;
  st.N = N;
  st.n = n;
  st.nnz = nnz;
  st.n_ops = (int)c->ops.size();
  double n0 = 0, nall = 0, z0 = 0, zall = 0;
  for (auto& op : c->ops) {
    if (op.jacobi) continue;
    st.max_levels_used = std::max(st.max_levels_used, op.h.nlev());
    n0 += op.h.L[0].A.n;
    z0 += op.h.L[0].A.nnz;
    for (auto& lv : op.h.L) {
      nall += lv.A.n;
      zall += lv.A.nnz;
    }
  }
  st.grid_complexity = n0 > 0 ? nall / n0 : 0;
  st.op_complexity = z0 > 0 ? zall / z0 : 0;
  double vbytes = 0;
  auto count_bytes = [&](auto& B) {
    for (const Step& s2 : c->steps) {
      if (s2.type == Step::INVERT && s2.batch >= 0) {
        int maxc = 1;
        for (int id : s2.ops) maxc = std::max(maxc, c->ops[id].count);
        vbytes += B[s2.batch].bytes_total * maxc;
      }
    }
  };
  if (mixed(c)) count_bytes(c->vb32);
  else count_bytes(c->vb64);
  double pbytes = vbytes;
  for (const Step& s2 : c->steps)
    if (s2.type != Step::INVERT) pbytes += s2.bytes;
  st.vcycle_bytes = vbytes;
  st.precond_bytes = pbytes;
  st.iter_bytes_base = sp_bytes(nnz, n, 8) + 16.0 * n + 4 * 8.0 * 2 * n + 16.0 * n;
  st.n_dropped = ndrop;
  st.n_jacobi_ops = c->n_jacobi;
  st.setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  c->ready = true;
}

// Right-preconditioned FGMRES(m) (Saad 1993) with modified Gram-Schmidt
// Arnoldi on the device; the small Hessenberg problem and its Givens rotations
// are solved on the host in FP64 from one device-to-host copy per iteration.
static int fgmres(mgd_ctx* c, const double* b, double* x, double tol, bool trans, int* iters, double* relres) {
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = c->s;
  int n = c->n, m = c->m;
  const Csr& A = trans ? c->AT : c->A;
  const Sell& AS = trans ? c->ATsell : c->Asell;
  double* hp = c->hpin;
  auto norm = [&](const double* v) {
    launch_norm2(n, v, c->partial, c->hbuf + 96, s);
    MGD_CUDA(cudaMemcpyAsync(hp + 200, c->hbuf + 96, sizeof(double), cudaMemcpyDeviceToHost, s));
    MGD_CUDA(cudaStreamSynchronize(s));
    c->prof.harvest();
    return std::sqrt(hp[200]);
  };
  auto spmv = [&](const double* in, double* out) {
    int id = c->prof.begin(s, 2);
    launch_spmv_f64(c->fmtMono, n, A.rp, A.ci, A.v, AS.sptr, AS.ci, AS.v, in, out, s);
    c->prof.end(id, 2, sp_bytes(A.nnz, n, 8) + 16.0 * n, s);
  };
  c->hist.clear();
  double bnorm = norm(b);
  *iters = 0;
  if (bnorm == 0.0) {
    MGD_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    MGD_CUDA(cudaStreamSynchronize(s));
    *relres = 0.0;
    return MGD_OK;
  }
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  auto Hm = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
  int it = 0, status = MGD_ENOCONV;
  bool broke = false;  // an Arnoldi breakdown ended the previous cycle
  for (;;) {
    int id = c->prof.begin(s, 2);
    launch_resid_f64(c->fmtMono, n, A.rp, A.ci, A.v, AS.sptr, AS.ci, AS.v, b, x, c->r, s);
    c->prof.end(id, 2, sp_bytes(A.nnz, n, 8) + 24.0 * n, s);
    double beta = norm(c->r);
    *relres = beta / bnorm;
    if (!std::isfinite(beta)) {
      status = MGD_ENAN;
      break;
    }
    if (beta <= tol * bnorm) {
      status = MGD_OK;
      break;
    }
    // h_{j+1,j} = 0 with a nonsingular Hessenberg matrix gives the exact
    // solution of the preconditioned system; if the true residual still misses
    // the tolerance, a restart from the same data cannot do better
    if (broke) {
      status = MGD_EBREAKDOWN;
      break;
    }
    if (it >= c->o.max_it) {
      status = MGD_ENOCONV;
      break;
    }
    // V_0 = r / beta  (scale_by_norm takes a squared norm)
    hp[201] = beta * beta;
    MGD_CUDA(cudaMemcpyAsync(c->hbuf + 101, hp + 201, sizeof(double), cudaMemcpyHostToDevice, s));
    launch_scale_by_norm(n, c->r, c->hbuf + 101, c->V, s);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int j = 0;
    while (j < m) {
      double* vj = c->V + (size_t)j * n;
      double* zj = c->Z + (size_t)j * n;
      precond_apply(c, vj, zj, trans);
      ++it;
      spmv(zj, c->w);
      int nv = j + 1;
      int aid = c->prof.begin(s, 3);
      // modified Gram-Schmidt: h in hbuf[0..j], ||w||^2 in hbuf[64], v_{j+1} = w / ||w||
      if (c->arn_nb > 0) {
        launch_arnoldi_coop(c->arn_nb, n, c->V, n, nv, c->w, c->hbuf, c->hbuf + 64, c->partial,
                            c->V + (size_t)(j + 1) * n, s);
      } else {
        // class 5: the j+1 fused Gram-Schmidt steps alone (32 n bytes each)
        int sid = -1;
        launch_mgs(
            n, c->V, n, nv, c->w, c->hbuf, c->hbuf + 64, c->partial, c->partial + kDotBlocks, s,
            [&] { sid = c->prof.begin(s, 5); }, [&] { c->prof.end(sid, 5, 32.0 * n * nv, s); });
        // the last step (index nv-1) ran backwards when nv-1 is odd: run the opposite way
        launch_scale_by_norm(n, c->w, c->hbuf + 64, c->V + (size_t)(j + 1) * n, s, ((nv - 1) & 1) ? 0 : 1);
      }
      c->prof.end(aid, 3, 8.0 * n * (4.0 * nv + 2.0 + 2.0), s);
      MGD_CUDA(cudaMemcpyAsync(hp, c->hbuf, 65 * sizeof(double), cudaMemcpyDeviceToHost, s));
      MGD_CUDA(cudaStreamSynchronize(s));
      c->prof.harvest();
      for (int i = 0; i <= j; ++i) Hm(i, j) = hp[i];
      double hn = std::sqrt(hp[64]);
      Hm(j + 1, j) = hn;
      for (int i = 0; i < j; ++i) {
        double t = cs[i] * Hm(i, j) + sn[i] * Hm(i + 1, j);
        Hm(i + 1, j) = -sn[i] * Hm(i, j) + cs[i] * Hm(i + 1, j);
        Hm(i, j) = t;
      }
      double h1 = Hm(j, j), h2 = Hm(j + 1, j);
      if (h2 == 0.0) {
        cs[j] = 1.0;
        sn[j] = 0.0;
      } else {
        double tt = std::sqrt(h1 * h1 + h2 * h2);
        cs[j] = h1 / tt;
        sn[j] = h2 / tt;
      }
      Hm(j, j) = cs[j] * h1 + sn[j] * h2;
      Hm(j + 1, j) = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      c->hist.push_back(std::fabs(g[j + 1]) / bnorm);
      ++j;
      if (hn == 0.0) broke = true;
      if (std::fabs(g[j]) <= tol * bnorm || hn == 0.0 || it >= c->o.max_it || !std::isfinite(g[j])) break;
    }
    // a zero on the diagonal of the rotated Hessenberg matrix: the small
    // least-squares problem is singular, no solution in this Krylov space;
    // x keeps its value
    bool singular = false;
    for (int i = 0; i < j; ++i)
      if (Hm(i, i) == 0.0) singular = true;
    if (singular) {
      status = MGD_EBREAKDOWN;
      break;
    }
    for (int i = j - 1; i >= 0; --i) {
      double sum = g[i];
      for (int k = i + 1; k < j; ++k) sum -= Hm(i, k) * y[k];
      y[i] = sum / Hm(i, i);
    }
    for (int i = 0; i < j; ++i) hp[100 + i] = y[i];
    MGD_CUDA(cudaMemcpyAsync(c->ybuf, hp + 100, sizeof(double) * j, cudaMemcpyHostToDevice, s));
    launch_vcomb(n, c->Z, n, j, c->ybuf, x, s);
  }
  MGD_CUDA(cudaStreamSynchronize(s));
  *iters = it;
  c->st.last_iters = it;
  c->st.last_relres = *relres;
  c->st.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (status != MGD_OK) {
    if (status == MGD_ENOCONV) c->err = "iteration cap reached";
    if (status == MGD_ENAN) c->err = "non-finite residual";
    if (status == MGD_EBREAKDOWN) c->err = "Arnoldi breakdown without reaching the tolerance";
  }
  return status;
}

// ------------------------------------------------------------------ C ABI
extern "C" {

int mgd_opts_default(mgd_opts* o) {
  if (!o) return MGD_EINVAL;
  memset(o, 0, sizeof(*o));
  o->theta_str = 0.25;
  o->max_coarse = 100;
  o->max_levels = 25;
  o->theta_wd = 0.9;
  o->theta_wc = 1e-2;
  o->sigma_wc = 0.5;
  o->inner_tol = 1e-2;
  o->inner_maxit = 100;
  o->nvcyc_group = 1;
  o->nvcyc_E = 1;
  o->nvcyc_I = 1;
  o->nvcyc_other = 1;
  o->jacobi_sweeps = 1;
  o->adaptive = 0;
  o->seed = 0;
  o->restart = 30;
  o->max_it = 1000;
  o->precision = 0;
  o->batched = 0;
  o->use_graph = 0;
  o->autotune = 1;
  o->keep_transpose = 0;
  o->fuse_rows = 0;
  o->interp_type = 0;
  o->pdl = 1;
  o->inner_mode = 0;
  o->smoother = 0;
  o->agg_levels = 0;
  o->arnoldi_resident = 1;
  o->opt4_steps = 0;
  return MGD_OK;
}

int mgd_create(mgd_ctx** out, const mgd_opts* o, void* stream) {
  if (!out) return MGD_EINVAL;
  *out = nullptr;
  mgd_ctx* c = new (std::nothrow) mgd_ctx();
  if (!c) return MGD_ENOMEM;
  if (o) c->o = *o;
  else mgd_opts_default(&c->o);
  const mgd_opts& q = c->o;
  if (q.max_coarse < 1 || q.max_coarse > 4096 || q.max_levels < 1 || q.restart < 1 || q.restart > 30 ||
      q.precision < 0 || q.precision > 1 || q.inner_mode < 0 || q.inner_mode > 1 || q.inner_maxit < 1 ||
      q.inner_maxit > 100000 || !(q.inner_tol >= 0.0) || q.nvcyc_group > 1000 || q.nvcyc_E > 1000 ||
      q.nvcyc_I > 1000 || q.nvcyc_other > 1000 || q.jacobi_sweeps > 1000 || q.smoother < 0 || q.smoother > 1 ||
      q.agg_levels < 0 || q.agg_levels > q.max_levels || q.arnoldi_resident < 0 || q.arnoldi_resident > 1 ||
      q.opt4_steps < 0 || q.opt4_steps > 1000) {
    delete c;
    return MGD_EINVAL;
  }
  c->s = (cudaStream_t)stream;
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return MGD_ECUDA;
  }
  try {
    c->pool.create(c->device);
  } catch (const Error& e) {
    delete c;
    return e.code;
  }
  c->ar.pool = c->pool.pool;
  c->ar.stream = c->s;
  *out = c;
  return MGD_OK;
}

int mgd_setup(mgd_ctx* c, int G, int N, int n, int nnz, const int* d_rowptr, const int* d_colidx,
              const double* d_vals, int kind) {
  return guarded(c, [&]() -> int {
    if (G < 1 || N < 1 || n != (G + 2) * N || nnz < n || !d_rowptr || !d_colidx || !d_vals || kind < 0 ||
        kind > MGD_BLT || G + 1 > kMaxTerms - 1)
      throw Error{MGD_EINVAL, "invalid sizes or kind"};
    const double rel_ms = free_setup_timed(c);
    c->G = G;
    c->N = N;
    c->n = n;
    c->nnz = nnz;
    c->kind = kind;
    do_setup(c, d_rowptr, d_colidx, d_vals);
    record_phase(c, SP_RELEASE, rel_ms);
    return MGD_OK;
  });
}

// Host arrays to the device in 32 MiB chunks spread over the context's copy
// streams (several copy engines at once), joined back into the context
// stream; the destination is stream-ordered memory of the context stream.
static void h2d_spread(mgd_ctx* c, void* dst, const void* src, size_t bytes, int& next) {
  const size_t chunk = (size_t)32 << 20;
  for (size_t o = 0; o < bytes; o += chunk) {
    cudaStream_t cs = c->s_copy[next++ % 4];
    MGD_CUDA(cudaMemcpyAsync((char*)dst + o, (const char*)src + o, std::min(chunk, bytes - o),
                             cudaMemcpyHostToDevice, cs));
  }
}

int mgd_setup_host(mgd_ctx* c, int G, int N, int n, int nnz, const int* h_rowptr, const int* h_colidx,
                   const double* h_vals, int kind) {
  return guarded(c, [&]() -> int {
    if (G < 1 || N < 1 || n != (G + 2) * N || nnz < n || !h_rowptr || !h_colidx || !h_vals || kind < 0 ||
        kind > MGD_BLT || G + 1 > kMaxTerms - 1)
      throw Error{MGD_EINVAL, "invalid sizes or kind"};
    for (auto& cs : c->s_copy)
      if (!cs) MGD_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    // the previous setup goes first; the host arrays are copied straight into
    // the new setup's arena, where they stay as the monolithic operator
    const double rel_ms = free_setup_timed(c);
    c->ar.stream = c->s;
    int* rp = c->ar.alloc<int>((size_t)n + 1);
    int* ci = c->ar.alloc<int>(nnz);
    double* v = c->ar.alloc<double>(nnz);
    struct CopyDrain {  // on any exit path the copies have ended before the arena can be released
      mgd_ctx* c;
      ~CopyDrain() {
        for (auto cs : c->s_copy)
          if (cs) cudaStreamSynchronize(cs);
      }
    } drain{c};
    auto th = std::chrono::steady_clock::now();
    struct Events {  // released on every exit path
      cudaEvent_t e[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
      ~Events() {
        for (auto x : e)
          if (x) cudaEventDestroy(x);
      }
    } ev;
    for (auto& e : ev.e) MGD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    MGD_CUDA(cudaEventRecord(ev.e[4], c->s));
    for (auto cs : c->s_copy) MGD_CUDA(cudaStreamWaitEvent(cs, ev.e[4], 0));
    int next = 0;
    h2d_spread(c, v, h_vals, sizeof(double) * (size_t)nnz, next);
    h2d_spread(c, ci, h_colidx, sizeof(int) * (size_t)nnz, next);
    h2d_spread(c, rp, h_rowptr, sizeof(int) * ((size_t)n + 1), next);
    for (int k = 0; k < 4; ++k) {
      MGD_CUDA(cudaEventRecord(ev.e[k], c->s_copy[k]));
      MGD_CUDA(cudaStreamWaitEvent(c->s, ev.e[k], 0));
    }
    MGD_CUDA(cudaStreamSynchronize(c->s));
    const double h2d_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - th).count();
    c->G = G;
    c->N = N;
    c->n = n;
    c->nnz = nnz;
    c->kind = kind;
    do_setup(c, rp, ci, v, true);
    record_phase(c, SP_H2D, h2d_ms);
    record_phase(c, SP_RELEASE, rel_ms);
    return MGD_OK;
  });
}

int mgd_update_values(mgd_ctx* c, const double* d_vals) {
  return guarded(c, [&]() -> int {
    if (!c->ready) throw Error{MGD_ESTATE, "no setup"};
    // keep the pattern of the current operator, replace the values, redo the setup
    Scratch sc(c->s);
    int* rp = sc.alloc<int>(c->n + 1);
    int* ci = sc.alloc<int>(c->nnz);
    double* v = sc.alloc<double>(c->nnz);
    MGD_CUDA(cudaMemcpyAsync(rp, c->A.rp, sizeof(int) * (c->n + 1), cudaMemcpyDeviceToDevice, c->s));
    MGD_CUDA(cudaMemcpyAsync(ci, c->A.ci, sizeof(int) * c->nnz, cudaMemcpyDeviceToDevice, c->s));
    MGD_CUDA(cudaMemcpyAsync(v, d_vals, sizeof(double) * c->nnz, cudaMemcpyDeviceToDevice, c->s));
    MGD_CUDA(cudaStreamSynchronize(c->s));
    const double rel_ms = free_setup_timed(c);
    do_setup(c, rp, ci, v);
    record_phase(c, SP_RELEASE, rel_ms);
    return MGD_OK;
  });
}

int mgd_solve(mgd_ctx* c, const double* d_b, double tol, double* d_x, int* iters, double* relres) {
  return guarded(c, [&]() -> int {
    if (!c->ready) throw Error{MGD_ESTATE, "solve before setup"};
    if (!d_b || !d_x || !(tol > 0)) throw Error{MGD_EINVAL, "invalid arguments"};
    int it = 0;
    double rr = 0;
    int r = fgmres(c, d_b, d_x, tol, false, &it, &rr);
    if (iters) *iters = it;
    if (relres) *relres = rr;
    return r;
  });
}

int mgd_solve_host(mgd_ctx* c, const double* h_b, double tol, double* h_x, int* iters, double* relres) {
  return guarded(c, [&]() -> int {
    if (!c->ready) throw Error{MGD_ESTATE, "solve before setup"};
    if (!h_b || !h_x || !(tol > 0)) throw Error{MGD_EINVAL, "invalid arguments"};
    MGD_CUDA(cudaMemcpyAsync(c->btmp, h_b, sizeof(double) * c->n, cudaMemcpyHostToDevice, c->s));
    MGD_CUDA(cudaMemcpyAsync(c->xtmp, h_x, sizeof(double) * c->n, cudaMemcpyHostToDevice, c->s));
    int it = 0;
    double rr = 0;
    int r = fgmres(c, c->btmp, c->xtmp, tol, false, &it, &rr);
    MGD_CUDA(cudaMemcpyAsync(h_x, c->xtmp, sizeof(double) * c->n, cudaMemcpyDeviceToHost, c->s));
    MGD_CUDA(cudaStreamSynchronize(c->s));
    if (iters) *iters = it;
    if (relres) *relres = rr;
    return r;
  });
}

int mgd_solve_transpose(mgd_ctx* c, const double* d_g, double tol, double* d_lambda, int* iters, double* relres) {
  return guarded(c, [&]() -> int {
    if (!c->ready) throw Error{MGD_ESTATE, "solve before setup"};
    if (!c->o.keep_transpose) throw Error{MGD_ESTATE, "setup without keep_transpose"};
    if (c->kind != MGD_AMG && c->kind != MGD_BD) throw Error{MGD_EINVAL, "transposed solve needs AMG or BD"};
    if (!d_g || !d_lambda || !(tol > 0)) throw Error{MGD_EINVAL, "invalid arguments"};
    int it = 0;
    double rr = 0;
    int r = fgmres(c, d_g, d_lambda, tol, true, &it, &rr);
    if (iters) *iters = it;
    if (relres) *relres = rr;
    return r;
  });
}

int mgd_grad_values(mgd_ctx* c, const double* d_x, const double* d_lambda, double* d_grad) {
  return guarded(c, [&]() -> int {
    if (!c->ready) throw Error{MGD_ESTATE, "no setup"};
    if (!d_x || !d_lambda || !d_grad) throw Error{MGD_EINVAL, "invalid arguments"};
    launch_grad_vals(c->n, c->A.rp, c->A.ci, d_x, d_lambda, d_grad, c->s);
    MGD_CUDA(cudaStreamSynchronize(c->s));
    return MGD_OK;
  });
}

int mgd_precond_apply(mgd_ctx* c, const double* d_v, double* d_z) {
  return guarded(c, [&]() -> int {
    if (!c->ready) throw Error{MGD_ESTATE, "no setup"};
    if (!d_v || !d_z) throw Error{MGD_EINVAL, "invalid arguments"};
    precond_apply(c, d_v, d_z, false);
    MGD_CUDA(cudaStreamSynchronize(c->s));
    c->prof.harvest();
    return MGD_OK;
  });
}

int mgd_precond_bench(mgd_ctx* c, const double* d_v, double* d_z, int count, double* ms_per_apply,
                      double* bytes_per_apply) {
  return guarded(c, [&]() -> int {
    if (!c->ready) throw Error{MGD_ESTATE, "no setup"};
    if (!d_v || !d_z || count < 1 || !ms_per_apply || !bytes_per_apply) throw Error{MGD_EINVAL, "invalid arguments"};
    cudaEvent_t e0, e1;
    MGD_CUDA(cudaEventCreate(&e0));
    MGD_CUDA(cudaEventCreate(&e1));
    float ms = 0.0f;
    try {
      precond_apply(c, d_v, d_z, false);  // warm
      MGD_CUDA(cudaEventRecord(e0, c->s));
      for (int k = 0; k < count; ++k) precond_apply(c, d_v, d_z, false);
      MGD_CUDA(cudaEventRecord(e1, c->s));
      MGD_CUDA(cudaEventSynchronize(e1));
      MGD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    } catch (...) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->prof.harvest();
    *ms_per_apply = (double)ms / count;
    *bytes_per_apply = c->st.precond_bytes;
    return MGD_OK;
  });
}

int mgd_get_stats(mgd_ctx* c, mgd_stats* s) {
  if (!c || !s) return MGD_EINVAL;
  *s = c->st;
  return MGD_OK;
}

int mgd_get_history(mgd_ctx* c, double* h, int cap, int* count) {
  if (!c || !count) return MGD_EINVAL;
  int k = std::min<int>(cap, (int)c->hist.size());
  for (int i = 0; i < k && h; ++i) h[i] = c->hist[i];
  *count = (int)c->hist.size();
  return MGD_OK;
}

int mgd_op_info(mgd_ctx* c, int op, int* kind, int* comp, int* nlevels, int* use_jacobi, int* coarse_lu) {
  if (!c || !c->ready || op < 0 || op >= (int)c->ops.size()) return MGD_EINVAL;
  InvOp& o = c->ops[op];
  if (kind) *kind = o.kind;
  if (comp) *comp = o.comp;
  if (nlevels) *nlevels = o.jacobi ? 0 : o.h.nlev();
  if (use_jacobi) *use_jacobi = o.jacobi;
  if (coarse_lu) *coarse_lu = o.jacobi ? 0 : o.h.coarse_lu;
  return MGD_OK;
}

int mgd_level_info(mgd_ctx* c, int op, int level, int* n, int* nnz, int* nnzP, int* ncoarse) {
  if (!c || !c->ready || op < 0 || op >= (int)c->ops.size()) return MGD_EINVAL;
  InvOp& o = c->ops[op];
  if (o.jacobi || level < 0 || level >= o.h.nlev()) return MGD_EINVAL;
  Level& lv = o.h.L[level];
  if (n) *n = lv.A.n;
  if (nnz) *nnz = lv.A.nnz;
  if (nnzP) *nnzP = level < o.h.nlev() - 1 ? lv.P.nnz : 0;
  if (ncoarse) *ncoarse = level < o.h.nlev() - 1 ? lv.nc : 0;
  return MGD_OK;
}

int mgd_op_cycles(mgd_ctx* c, int op, long long* cycles) {
  return guarded(c, [&]() -> int {
    if (!c->ready || op < 0 || op >= (int)c->ops.size() || !cycles) throw Error{MGD_EINVAL, "bad operator"};
    const InvOp& o = c->ops[op];
    long long n = 0;
    if (!o.jacobi) {
      for (const Step& st : c->steps) {
        if (st.type != Step::INVERT) continue;
        if (std::find(st.ops.begin(), st.ops.end(), op) == st.ops.end()) continue;
        n += (long long)o.count * c->napplyT;  // the transposed apply runs the fixed count
        auto it = std::find(st.loop_ops.begin(), st.loop_ops.end(), op);
        if (st.loop && it != st.loop_ops.end()) {
          long long t = 0;
          MGD_CUDA(cudaMemcpyAsync(&t, st.total + (it - st.loop_ops.begin()), sizeof(t), cudaMemcpyDeviceToHost,
                                   c->s));
          MGD_CUDA(cudaStreamSynchronize(c->s));
          n += t;
        } else {
          n += (long long)o.count * c->napply;
        }
      }
    }
    *cycles = n;
    return MGD_OK;
  });
}

int mgd_level_keys(mgd_ctx* c, int op, int level, int* nkeys, int* h_key) {
  return guarded(c, [&]() -> int {
    if (!c->ready || op < 0 || op >= (int)c->ops.size() || !nkeys) throw Error{MGD_EINVAL, "bad operator"};
    InvOp& o = c->ops[op];
    if (o.jacobi || level < 0 || level >= o.h.nlev()) throw Error{MGD_EINVAL, "bad level"};
    Level& lv = o.h.L[level];
    *nkeys = lv.nk;
    if (h_key && lv.nk > 0) {
      MGD_CUDA(cudaMemcpyAsync(h_key, lv.key, sizeof(int) * lv.A.n, cudaMemcpyDeviceToHost, c->s));
      MGD_CUDA(cudaStreamSynchronize(c->s));
    }
    return MGD_OK;
  });
}

int mgd_level_export(mgd_ctx* c, int op, int level, int* h_rp, int* h_ci, double* h_v, signed char* h_cf,
                     int* h_prp, int* h_pci, double* h_pv) {
  return guarded(c, [&]() -> int {
    if (!c->ready || op < 0 || op >= (int)c->ops.size()) throw Error{MGD_EINVAL, "bad operator"};
    InvOp& o = c->ops[op];
    if (o.jacobi || level < 0 || level >= o.h.nlev()) throw Error{MGD_EINVAL, "bad level"};
    Level& lv = o.h.L[level];
    bool last = level == o.h.nlev() - 1;
    auto cp = [&](void* dst, const void* src, size_t bytes) {
      if (dst && src && bytes) MGD_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c->s));
    };
    cp(h_rp, lv.A.rp, sizeof(int) * (lv.A.n + 1));
    cp(h_ci, lv.A.ci, sizeof(int) * lv.A.nnz);
    cp(h_v, lv.A.v, sizeof(double) * lv.A.nnz);
    if (!last) {
      cp(h_cf, lv.CF, lv.A.n);
      cp(h_prp, lv.P.rp, sizeof(int) * (lv.A.n + 1));
      cp(h_pci, lv.P.ci, sizeof(int) * lv.P.nnz);
      cp(h_pv, lv.P.v, sizeof(double) * lv.P.nnz);
    }
    MGD_CUDA(cudaStreamSynchronize(c->s));
    return MGD_OK;
  });
}

int mgd_block_vector(mgd_ctx* c, int which, int comp, int comp2, double* h_out) {
  return guarded(c, [&]() -> int {
    if (!c->ready || c->kind == MGD_AMG || !h_out || comp < 0 || comp >= c->G + 2)
      throw Error{MGD_EINVAL, "no block data"};
    const double* src = nullptr;
    int nc = c->G + 2;
    if (which == 0 && !c->bd.p.empty()) src = c->bd.p[comp];
    if (which == 1) src = c->bd.diag[comp];
    if (which == 2 && comp2 >= 0 && comp2 < nc) src = c->bd.d[comp * nc + comp2];
    if (!src) throw Error{MGD_EINVAL, "vector absent"};
    MGD_CUDA(cudaMemcpyAsync(h_out, src, sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->s));
    MGD_CUDA(cudaStreamSynchronize(c->s));
    return MGD_OK;
  });
}

int mgd_coupling_dropped(mgd_ctx* c, int a, int b) {
  if (!c || !c->ready || c->bd.dropped.empty()) return 0;
  int nc = c->G + 2;
  if (a < 0 || b < 0 || a >= nc || b >= nc) return 0;
  return c->bd.dropped[a * nc + b];
}

int mgd_profile_enable(mgd_ctx* c, int mask) {
  return guarded(c, [&]() -> int {
    MGD_CUDA(cudaStreamSynchronize(c->s));
    c->prof.harvest();
    bool changed = c->prof.mask != (unsigned)mask;
    c->prof.on = mask != 0;
    c->prof.mask = (unsigned)mask;
    c->prof.reset();
    // the captured graph carries its own event nodes: re-capture for the new mask
    if (changed && c->ready && c->o.use_graph) capture_graph(c);
    return MGD_OK;
  });
}

int mgd_profile_read(mgd_ctx* c, int cls, long long* launches, double* ms, double* bytes) {
  return guarded(c, [&]() -> int {
    if (cls < 0 || cls >= Profiler::kClasses) throw Error{MGD_EINVAL, "bad class"};
    MGD_CUDA(cudaStreamSynchronize(c->s));
    c->prof.harvest();
    long long nl = c->prof.n[cls];
    double t = c->prof.ms[cls], by = c->prof.bytes[cls];
    if (cls == 1) {  // every V-cycle kernel
      nl += c->prof.n[0];
      t += c->prof.ms[0];
      by += c->prof.bytes[0];
    }
    if (launches) *launches = nl;
    if (ms) *ms = t;
    if (bytes) *bytes = by;
    return MGD_OK;
  });
}

int mgd_profile_read_fp64(mgd_ctx* c, int cls, double* fp64_ops) {
  return guarded(c, [&]() -> int {
    if (cls < 0 || cls >= Profiler::kClasses || !fp64_ops) throw Error{MGD_EINVAL, "bad class or null output"};
    MGD_CUDA(cudaStreamSynchronize(c->s));
    c->prof.harvest();
    double f = c->prof.fp64[cls];
    if (cls == 1) f += c->prof.fp64[0];
    *fp64_ops = f;
    return MGD_OK;
  });
}

int mgd_fp64_issue_rate(void* stream, double* lane_ops_per_s) {
  if (!lane_ops_per_s) return MGD_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  try {
    *lane_ops_per_s = measure_fp64_rate(s);
  } catch (const Error&) {
    cudaGetLastError();
    return MGD_ECUDA;
  }
  return MGD_OK;
}

int mgd_check_conversions(void* stream, long long* mismatches) {
  if (!mismatches) return MGD_EINVAL;
  try {
    *mismatches = check_conversions(static_cast<cudaStream_t>(stream));
  } catch (const Error&) {
    cudaGetLastError();
    return MGD_ECUDA;
  }
  return MGD_OK;
}

const char* mgd_last_error(mgd_ctx* c) { return c ? c->err.c_str() : "null context"; }

int mgd_plan_info(mgd_ctx* c, int batch, int level, int* nbatches, int* depth, int* nsub, int* maxrows, int* fmtA,
                  int* fmtR, int* fmtP, int* tail) {
  if (!c || !c->ready) return MGD_EINVAL;
  bool m = mixed(c);
  int nb = m ? (int)c->vb32.size() : (int)c->vb64.size();
  if (nbatches) *nbatches = nb;
  if (batch < 0 || batch >= nb) return MGD_EINVAL;
  auto fill = [&](auto& vb) -> int {
    if (depth) *depth = vb.depth;
    if (tail) *tail = vb.tail_level;
    if (level < 0 || level >= vb.depth) return MGD_EINVAL;
    auto& lp = vb.plan[level];
    if (nsub) *nsub = lp.ndown;
    if (maxrows) *maxrows = lp.maxn;
    if (fmtA) *fmtA = lp.fmtA;
    if (fmtR) *fmtR = lp.fmtR;
    if (fmtP) *fmtP = lp.fmtP;
    return MGD_OK;
  };
  return m ? fill(c->vb32[batch]) : fill(c->vb64[batch]);
}

int mgd_setup_phases(mgd_ctx* c, double* h_ms, int n) {
  if (!c || !h_ms || n < 0) return MGD_EINVAL;
  std::lock_guard<std::mutex> lk(c->phases.mu);
  for (int k = 0; k < n && k < SP_COUNT; ++k) h_ms[k] = c->phases.ms[k];
  return MGD_OK;
}

long long mgd_kernel_launches(void) { return __atomic_load_n(&g_kernel_launches, __ATOMIC_RELAXED); }

void mgd_destroy(mgd_ctx* c) {
  if (!c) return;
  free_setup(c);
  if (c->s_body) cudaStreamDestroy(c->s_body);
  for (auto cs : c->s_copy)
    if (cs) cudaStreamDestroy(cs);
  if (c->hpin) cudaFreeHost(c->hpin);
  c->pool.destroy();
  delete c;
}

}  // extern "C"
