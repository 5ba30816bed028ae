/*
 * mgdamg.h -- C ABI of the GB300 (sm_103a) solver for the (G+2)x(G+2)-block
 * linear systems of multi-group radiation diffusion (Eq. 2.2): classical-AMG
 * block preconditioners (monolithic AMG, Section 3.1; PCTL, Section 3.3;
 * Schur1 and Schur2, Section 3.4; block-diagonal and block lower-triangular,
 * the Remarks of Section 3.6) inside right-preconditioned FGMRES(m).
 *
 * Conventions for every entry point:
 *   - "d_" pointers are device pointers (CUDA global memory on the device that
 *     was current at mgd_create), "h_" pointers are host pointers.
 *   - Input arrays stay owned by the caller and are only read during the call;
 *     the library copies what it keeps.  Output arrays are caller-owned and
 *     must hold the stated number of elements.
 *   - All device work is issued on the CUDA stream given to mgd_create.  A
 *     call returns after its results are complete on that stream, unless its
 *     comment says otherwise.
 *   - Return value 0 is success; otherwise one of the MGD_E* codes below, with
 *     a message from mgd_last_error.  No C++ exception crosses this boundary.
 *   - Indices are 0-based int32.  The matrix is CSR with strictly increasing
 *     column indices inside each row, in block-major order: unknown (a, k) of
 *     component a in cell k is row/column a*N + k, components 0..G-1 are the
 *     radiation groups, G is the electron and G+1 the ion temperature.
 *     Off-block entries must couple the same cell (the D_ab are diagonal).
 */
#ifndef MGDAMG_H
#define MGDAMG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mgd_ctx mgd_ctx; /* opaque, library-owned */

/* preconditioner kinds */
enum {
  MGD_AMG = 0,    /* one classical-AMG V(1,1) cycle on the whole system (Section 3.1) */
  MGD_PCTL = 1,   /* physical-variable-based two-level scheme (Section 3.3, Eq. 3.3) */
  MGD_SCHUR1 = 2, /* five-stage block Schur complement, Eq. 3.1 with C_R ~ diag(C_g) (Section 3.4) */
  MGD_SCHUR2 = 3, /* three-stage approximate block factorisation, Eq. 3.2 (Section 3.4) */
  MGD_BD = 4,     /* block diagonal (Remark, Section 3.6) */
  MGD_BLT = 5     /* block lower triangular (Remark, Section 3.6) */
};

/* status codes */
enum {
  MGD_OK = 0,
  MGD_EINVAL = 1,      /* bad argument, size, layout, unsorted/duplicate columns, non-positive diagonal */
  MGD_ENOCONV = 2,     /* iteration cap reached; x holds the last iterate */
  MGD_EBREAKDOWN = 3,  /* Arnoldi breakdown (h_{j+1,j} = 0) and the tolerance still unmet, or a singular
                          Hessenberg least-squares problem (x then keeps its value) */
  MGD_ESINGULAR = 4,   /* zero pivot in the coarsest-level elimination */
  MGD_ENAN = 5,        /* non-finite residual */
  MGD_ETIMEOUT = 6,    /* reserved, never returned: no kernel of this library waits on a flag that
                          another launch writes; its grid-wide barriers run in cooperative launches,
                          whose co-residency the runtime guarantees, and every device-controlled loop
                          has a trip cap */
  MGD_ECUDA = 7,       /* CUDA runtime error */
  MGD_ENOMEM = 8,      /* device allocation failed */
  MGD_ESTATE = 9       /* call out of order (e.g. solve before setup) */
};

typedef struct mgd_opts {
  double theta_str;       /* strength threshold, Section 3.1: 0.25 */
  int max_coarse;         /* coarsest level solved by elimination when it has <= this many rows: 100 */
  int max_levels;         /* 25 */
  double theta_wd;        /* Definition 2 threshold: 0.9 */
  double theta_wc;        /* Definition 1 threshold: 1e-2 */
  double sigma_wc;        /* Section 3.6 switch criterion: 0.5 */
  double inner_tol;       /* option #3 accuracy (Sections 3.4-3.5, Section 4: 1e-2) for the PCTL p_a and, when
                             inner_mode, for the inverses listed there */
  int inner_maxit;        /* option #3 cycle cap: 100 (1 .. 100000) */
  int nvcyc_group;        /* option #2 V-cycles per inverse of a group operator: 1 */
  int nvcyc_E;            /* ... of an E operator: 1 */
  int nvcyc_I;            /* ... of an I operator: 1 */
  int nvcyc_other;        /* ... of the monolithic or PCTL coarse operator: 1 */
  int jacobi_sweeps;      /* option #1 sweeps: 1 */
  int adaptive;           /* 1: Section 3.6 coupling drops and the Section 3.5 option #1/#2 choice */
  unsigned long long seed;/* PMIS weight seed */
  int restart;            /* FGMRES restart length m: 30 */
  int max_it;             /* cap on preconditioner applications per solve: 1000 */
  int precision;          /* 0: FP64 V-cycles; 1: FP32 V-cycles (storage and arithmetic) inside FP64 FGMRES */
  int batched;            /* 1: independent V-cycles of a stage run as one launch per level and phase */
  int use_graph;          /* 1: the preconditioner apply is replayed from a captured CUDA graph */
  int autotune;           /* 1: time sparse-kernel variants per level at setup and keep the fastest; the
                             decisions are cached per process by hierarchy shape and, when the environment
                             variable MGD_TUNE_CACHE names a file, read from and written to that file, so
                             that another process (a profiler run, the next job) runs the same plan */
  int keep_transpose;     /* 1: keep A_l^T per level so that mgd_solve_transpose can run */
  int fuse_rows;          /* levels below level 0 whose subsystems all have <= fuse_rows rows run, with every
                             coarser level, in one thread-block-cluster launch per V-cycle; 0: chosen by the
                             autotuner (not fused when autotune is off); -1: never */
  int interp_type;        /* 0: classical modified interpolation (Section 3.1); 1: extended+i (distance-two
                             classical interpolation, De Sterck, Falgout, Nolting, Yang 2008) */
  int pdl;                /* 1: solve kernels use programmatic dependent launch (each waits on its predecessor
                             in-kernel, so launch latency overlaps the previous kernel); 0: plain launches */
  int inner_mode;         /* 1: option #3 (Section 3.5) inside the preconditioner for the Schur-type inverses
                             C_E, C_g (Schur1), S_g, S_I (Schur2) and the PCTL block inverses A_a: x = 0, then
                             x += V(rhs - A x) until ||rhs - A x|| <= inner_tol ||rhs|| or inner_maxit cycles.
                             The loop runs on the device (a conditional CUDA graph node when use_graph); the
                             transposed apply keeps the fixed cycle counts.  0: option #2 (default) */
  int smoother;           /* 0: l1-Jacobi pre- and post-smoothing (default); 1: Section 3.1's Gauss-Seidel in
                             C/F order as multicolour Gauss-Seidel: the points of each level are coloured by
                             Jones-Plassmann rounds on the symmetrised graph of A_l (weights from the seeded
                             counter generator, stream 2000 + level); pre-smoothing sweeps the C colours then
                             the F colours, post-smoothing the same classes in the opposite order; each sweep
                             updates x_i += (b_i - (A x)_i) / a_ii for its (mutually uncoupled) points */
  int agg_levels;         /* levels, from the finest, coarsened aggressively (Section 3.1): a second strength +
                             PMIS pass (weight stream 1100 + level) on A1 = P1^T A P1, which is not kept as a
                             level, chooses the final C points among the first pass's; P = P1 P2 (two-stage
                             interpolation, each stage of interp_type).  0: none (default); at most max_levels */
  int arnoldi_resident;   /* 1 (default): each FGMRES orthogonalisation runs as one cooperative grid that keeps the
                             new Krylov vector in shared memory (one block per SM; used when n fits, else 0);
                             0: one streaming kernel per basis vector.  Same modified Gram-Schmidt either way */
  int opt4_steps;         /* option #4 (Section 3.5).  0 (default): off.  K in 1..1000: the Schur complement
                             whose inner inverse is one block -- S_I = A_I - D_IE A_E^-1 D_EI of Schur2 and
                             C_E = A_E - D_EI A_I^-1 D_IE of Schur1 -- is inverted by K steps of
                             w(0) = 0, w(k+1) = A_a^-1 (q + D_ab A_b^-1 D_ba w(k)), with the AMG inverses
                             (option #2) of the plain blocks A_a, A_b in place of S_I-hat / C_E-hat.  Forward
                             apply only (the transposed solve is AMG/BD only) */
} mgd_opts;

/* Fill *o with the defaults listed above.  Returns MGD_EINVAL if o is NULL. */
int mgd_opts_default(mgd_opts *o);

/* Create a context bound to the current CUDA device and to `stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the
 * handle; destroy it with mgd_destroy. */
int mgd_create(mgd_ctx **out, const mgd_opts *o, void *stream);

/* Setup phase (Section 3.1 setup; Sections 3.3-3.6 block operators):
 * G groups, N cells, n = (G+2)*N unknowns, nnz entries; d_rowptr[n+1],
 * d_colidx[nnz], d_vals[nnz] on the device.  Validates the layout (MGD_EINVAL
 * on failure; MGD_ENAN when a value is not finite),  extracts the blocks and couplings, applies the adaptive rules
 * when opts.adaptive, builds every AMG hierarchy on the device (strength,
 * PMIS, classical modified interpolation, Galerkin RAP, l1 diagonals, dense
 * coarsest inverse) and prepares the solve.  Replaces any previous setup. */
int mgd_setup(mgd_ctx *c, int G, int N, int n, int nnz, const int *d_rowptr, const int *d_colidx,
              const double *d_vals, int kind);

/* As mgd_setup with the CSR arrays in host memory: h_rowptr[n+1],
 * h_colidx[nnz], h_vals[nnz] are copied to the device (in 32 MiB chunks over
 * four copy streams, so several copy engines run at once; page-locked host
 * memory gives the full host-to-device bandwidth, pageable memory is staged by
 * the driver) straight into the device memory the setup keeps as its copy of
 * the operator, after the previous setup has been released, then set up
 * exactly as mgd_setup does.  The host arrays are only read, and may be reused
 * once the call returns.  Same errors as mgd_setup. */
int mgd_setup_host(mgd_ctx *c, int G, int N, int n, int nnz, const int *h_rowptr, const int *h_colidx,
                   const double *h_vals, int kind);

/* Same sparsity pattern, new values d_vals[nnz]: re-runs the whole numeric
 * setup (the coarse patterns may change with the values). */
int mgd_update_values(mgd_ctx *c, const double *d_vals);

/* Solve A x = b by FGMRES(restart) preconditioned on the right, stopping when
 * ||b - A x||_2 <= tol ||b||_2 (Section 4).  d_b[n] in, d_x[n] in: initial
 * guess, out: solution.  *iters = preconditioner applications, *relres = final
 * true relative residual.  Returns MGD_ENOCONV if max_it is reached,
 * MGD_ENAN when a residual norm is not finite (e.g. a NaN in b or in the
 * values), MGD_EBREAKDOWN as described with the status codes; a happy
 * breakdown that meets the tolerance returns MGD_OK. */
int mgd_solve(mgd_ctx *c, const double *d_b, double tol, double *d_x, int *iters, double *relres);

/* As mgd_solve with host buffers h_b[n], h_x[n] (x: initial guess in,
 * solution out); copies in and out on the context's stream. */
int mgd_solve_host(mgd_ctx *c, const double *h_b, double tol, double *h_x, int *iters, double *relres);

/* Adjoint solve A^T lambda = g with the transposed preconditioner (the V-cycle
 * run with A_l^T, the same P, R and smoother, and the transposed coarsest
 * solve).  Needs opts.keep_transpose and kind MGD_AMG or MGD_BD. */
int mgd_solve_transpose(mgd_ctx *c, const double *d_g, double tol, double *d_lambda, int *iters,
                        double *relres);

/* Gradient of a loss with respect to the stored values of A, given x = A^{-1} b
 * and lambda = A^{-T} dL/dx: d_grad[k] = -lambda[row(k)] * x[col(k)], k < nnz. */
int mgd_grad_values(mgd_ctx *c, const double *d_x, const double *d_lambda, double *d_grad);

/* One application z = M^{-1} v of the preconditioner (d_v[n], d_z[n]). */
int mgd_precond_apply(mgd_ctx *c, const double *d_v, double *d_z);

/* Measurement service (Section 4's preconditioner applied back to back, as
 * the V-cycle bandwidth of the timing plan needs): z = M^{-1} v applied
 * `count` times on the context's stream with no synchronisation between
 * applies (graph replays when use_graph), timed by two CUDA events.
 * *ms_per_apply = elapsed / count; *bytes_per_apply = the algorithmic bytes
 * of one apply (its V-cycles and block updates, as mgd_stats.precond_bytes).
 * d_v[n], d_z[n] device buffers.  MGD_EINVAL for count < 1 or NULL pointers,
 * MGD_ESTATE before setup. */
int mgd_precond_bench(mgd_ctx *c, const double *d_v, double *d_z, int count, double *ms_per_apply,
                      double *bytes_per_apply);

/* Statistics of the current setup. */
typedef struct mgd_stats {
  int kind, G, N, n, nnz;
  int n_ops;                  /* number of scalar operators inverted by the preconditioner */
  int max_levels_used;        /* deepest hierarchy */
  double grid_complexity;     /* sum over operators and levels of n_l / sum of n_0 */
  double op_complexity;       /* sum of nnz(A_l) / sum of nnz(A_0) */
  double setup_ms;            /* wall time of the last mgd_setup */
  double solve_ms;            /* wall time of the last solve */
  int last_iters;
  double last_relres;
  double vcycle_bytes;        /* algorithmic HBM bytes of one preconditioner apply (V-cycles only) */
  double precond_bytes;       /* algorithmic bytes of one preconditioner apply including block updates */
  double iter_bytes_base;     /* bytes of one FGMRES iteration outside the preconditioner, for j = 0 */
  int n_dropped;              /* couplings dropped by the Section 3.6 rule */
  int n_jacobi_ops;           /* operators approximated by option #1 */
} mgd_stats;
int mgd_get_stats(mgd_ctx *c, mgd_stats *s);

/* Residual history of the last solve: h_hist[k] = Arnoldi estimate of the
 * relative residual after preconditioner application k+1 (k < *count). */
int mgd_get_history(mgd_ctx *c, double *h_hist, int cap, int *count);

/* Introspection of operator `op` (index into the preconditioner's operator
 * list, see mgd_op_info) for the parity tests. */
int mgd_op_info(mgd_ctx *c, int op, int *kind, int *comp, int *nlevels, int *use_jacobi, int *coarse_lu);
int mgd_level_info(mgd_ctx *c, int op, int level, int *n, int *nnz, int *nnzP, int *ncoarse);
/* *cycles = V-cycles (option #2/#3) applied by the inverse of operator `op`
 * since its setup, forward and transposed applies together (0 for an
 * option #1 Jacobi inverse).  Synchronises the context's stream (the option #3 counts
 * live on the device).  MGD_EINVAL for a bad op or NULL cycles. */
int mgd_op_cycles(mgd_ctx *c, int op, long long *cycles);
/* Gauss-Seidel order of level `level` of operator `op` (smoother 1): *nkeys =
 * number of sweeps; h_key[n] (host, may be NULL) = sweep index of each point.
 * *nkeys = 0 on the coarsest level or with the l1-Jacobi smoother. */
int mgd_level_keys(mgd_ctx *c, int op, int level, int *nkeys, int *h_key);
/* Copy level `level` of operator `op` to host buffers (any may be NULL):
 * A_l as h_rp[n+1], h_ci[nnz], h_v[nnz]; C/F splitting h_cf[n] (1 = C,
 * -1 = F; absent on the coarsest level); P_l as h_prp[n+1], h_pci[nnzP],
 * h_pv[nnzP]. */
int mgd_level_export(mgd_ctx *c, int op, int level, int *h_rp, int *h_ci, double *h_v, signed char *h_cf,
                     int *h_prp, int *h_pci, double *h_pv);
/* Block-level vectors (host copies, N entries): which = 0: PCTL p_a of
 * component comp; 1: diagonal of A_comp; 2: coupling D_{comp,comp2}. Returns
 * MGD_EINVAL when absent. */
int mgd_block_vector(mgd_ctx *c, int which, int comp, int comp2, double *h_out);
/* 1 if coupling D_{a,b} was dropped by the Section 3.6 rule. */
int mgd_coupling_dropped(mgd_ctx *c, int a, int b);

/* Host wall time (ms) of the phases of the last mgd_setup, h_ms[0..n-1]:
 * 0 strength, 1 PMIS, 2 interpolation, 3 transpose, 4 A P, 5 R (A P),
 * 6 level finalisation (diagonals, layouts, copies), 7 coarsest inverse --
 * these eight summed over every hierarchy (built concurrently, so they can
 * exceed the wall time) -- then 8 validation, 9 block extraction, 10 all
 * hierarchies (wall), 11 PCTL vectors and coarse operator, 12 launch program,
 * batches and autotuning, 13 Krylov storage and graph capture, 14 Gauss-Seidel
 * colouring (summed), 15 host-to-device copies (mgd_setup_host), 16 release of
 * the previous setup's device memory and graph. */
int mgd_setup_phases(mgd_ctx *c, double *h_ms, int n);

/* Launch plan of the V-cycle batches: *nbatches batches (independent V-cycles
 * launched together); for batch `batch` and level `level`, the number of
 * subsystems descending through that level, the largest row count, and the
 * autotuned layouts of the operator / restriction / prolongation kernels
 * (0 = SELL-32, 1..6 = CSR with 1, 2, 4, 8, 16, 32 threads per row, 7 / 8 =
 * SELL-32 with a thread on 2 / 4 slices, 9 / 10 = CSR with a thread on one
 * row of each of 2 / 4 adjacent 32-row groups); *tail =
 * first level handled by the fused coarse-level kernel (depth if none). */
int mgd_plan_info(mgd_ctx *c, int batch, int level, int *nbatches, int *depth, int *nsub, int *maxrows, int *fmtA,
                  int *fmtR, int *fmtP, int *tail);

/* Kernel timing for the roofline: CUDA events bracket every launch of the
 * kernel classes selected by the bit mask (bit k = class k; 0 turns timing
 * off, -1 selects all) on the context's stream.  Classes: 0 = level-0
 * smoothing+residual kernels of the V-cycle, 1 = the other V-cycle kernels,
 * 2 = the FGMRES operator SpMV and residual, 3 = Arnoldi vector kernels,
 * 4 = block-level updates of the block preconditioners, 5 = the fused
 * modified Gram-Schmidt steps of the streaming orthogonalisation alone
 * (j+1 launches per Arnoldi step, 32 n bytes each; inside class 3).  The read call
 * synchronises the stream and returns, for class cls (cls = 1 also counts
 * class 0, i.e. every V-cycle kernel), the launch count, the summed device
 * time and the summed algorithmic bytes.  V-cycle launches are also counted
 * under detail classes: 16 + 4*level + phase (phase 0 pre-smoothing +
 * residual, 1 restriction, 2 prolongation, 3 post-smoothing), 400 + level for
 * coarsest-level solves, 15 for the fused coarse-level kernel.  With opts.use_graph the selected
 * kernels are bracketed by event nodes inside the captured graph (the graph is
 * captured again when the mask changes), so timing does not change how the
 * preconditioner is launched. */
int mgd_profile_enable(mgd_ctx *c, int mask);
int mgd_profile_read(mgd_ctx *c, int cls, long long *launches, double *ms, double *bytes);
/* The algorithmic FP64 lane operations of the launches class cls recorded
 * (same classes and synchronisation as mgd_profile_read): one per nonzero and
 * two per row for the l1-Jacobi smoothing + residual kernels (k_pre, k_post),
 * one more per row for a stalled coarsest level's first sweep; zero for
 * FP32 V-cycles, Gauss-Seidel levels and the other kernels.  Together with
 * mgd_fp64_issue_rate it places the level-0 kernels against the FP64 issue
 * limit, which on GB300 is as low as the HBM limit for one multiply-add per
 * 12 bytes.  MGD_EINVAL for a bad class or a null output. */
int mgd_profile_read_fp64(mgd_ctx *c, int cls, double *fp64_ops);
/* Measures the device's FP64 multiply-add rate on `stream` (the current
 * device; a CUDA stream handle or NULL): two launches of 4 x SMs blocks of 512
 * threads, each thread running four independent chains of 4096 fused
 * multiply-adds, the second launch timed with CUDA events.  Writes lane
 * operations per second (every lane active) to *lane_ops_per_s.  Needs no
 * context; allocates ~2.5 MB stream-ordered and frees it.  MGD_EINVAL for a
 * null output, MGD_ECUDA when a CUDA call fails. */
int mgd_fp64_issue_rate(void *stream, double *lane_ops_per_s);
/* Self-check of the binary32 <-> binary64 conversions that the block updates
 * of the FP32-V-cycle form (precision = 1) do on the integer pipe (IEEE
 * 754-2008 formats, round to nearest even) against the hardware conversions,
 * on `stream` (the current device; a CUDA stream handle or NULL): every
 * binary32 pattern widened and narrowed back, and for every finite binary32
 * value the binary64 tie halfway to the next binary32 and that tie's two
 * binary64 neighbours narrowed.  Writes the number of differing results to
 * *mismatches (NaN results compare as equal when both are NaN).  Needs no
 * context; about 0.1 s; allocates 8 bytes stream-ordered and frees it.
 * MGD_EINVAL for a null output, MGD_ECUDA when a CUDA call fails. */
int mgd_check_conversions(void *stream, long long *mismatches);

/* Largest n accepted by mgd_relres_noalloc (its fixed work array holds n
 * doubles plus 1216 partial sums: about 4 MiB per GPU, kept until exit). */
#define MGD_NOALLOC_MAX_N (1 << 19)

/* True relative residual without any device allocation.  The paper has no
 * counterpart: this is a service for callers that cannot call cudaMalloc
 * (an application whose allocator owns the device, a loop with a fixed,
 * audited memory footprint).
 *
 * Computes r = b - A x for the CSR matrix d_rowptr[n+1], d_colidx, d_vals
 * (device pointers, any sparsity, int32 indices, FP64 values; not checked on
 * the device) and d_b[n], d_x[n], and writes d_out[0] = ||r||_2,
 * d_out[1] = ||b||_2, d_out[2] = ||r||_2 / ||b||_2 (0 when b = 0) into the
 * caller's device buffer d_out[3].  This is the quantity mgd_solve reports
 * as *relres.  Work runs on `stream` (a cudaStream_t, NULL = legacy default
 * stream); the call synchronises that stream before it returns.
 *
 * Work space is one fixed device array inside the library, not memory from
 * cudaMalloc.  CUDA loads device code lazily by default, so the first call
 * on a device may make the driver load this code and reserve the array
 * (about 4 MiB); after that no call allocates or frees device memory.
 * n < 1 or n > MGD_NOALLOC_MAX_N, or a null pointer, returns MGD_EINVAL; a
 * CUDA error of this call's launches returns MGD_ECUDA (an error left
 * pending by earlier work is cleared first, not reported).  The first call
 * on each device looks up that array's device address (once per device, with
 * that device current).  All calls share the array: calls that overlap on the
 * GPU (other streams, other threads) race and must be serialised by the
 * caller.  Nothing from an earlier call is read back. */
int mgd_relres_noalloc(int n, const int *d_rowptr, const int *d_colidx, const double *d_vals, const double *d_b,
                       const double *d_x, double *d_out, void *stream);

/* Kernels this library has launched in the calling process so far (a graph
 * replay counts each of its kernel nodes); a monotone counter for checking
 * that work ran on the device. */
long long mgd_kernel_launches(void);

const char *mgd_last_error(mgd_ctx *c);
void mgd_destroy(mgd_ctx *c);

#ifdef __cplusplus
}
#endif
#endif
