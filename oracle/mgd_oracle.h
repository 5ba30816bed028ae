/*
 * mgd_oracle.h -- plain, slow, single-threaded FP64 CPU oracle of classical-AMG
 * block preconditioners inside right-preconditioned FGMRES for the
 * (G+2)x(G+2)-block radiation-diffusion system (Eq. 2.2).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library; the product path never
 * does.  It shares no code with the CUDA library.
 *
 * Every function follows the paper's definitions in the paper's order; where
 * the paper is silent the reading used is stated beside the function.
 */
#ifndef MGD_ORACLE_H
#define MGD_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct or_csr {
  int n, m, nnz;          /* rows, columns, nonzeros */
  int *rp, *ci;           /* row pointer [n+1], sorted column indices [nnz] */
  double *v;              /* values [nnz] */
} or_csr;

typedef struct or_opts {
  double theta_str;       /* strength threshold, Section 3.1: 0.25 */
  int max_coarse;         /* coarsest level size solved by elimination: 100 */
  int max_levels;         /* 25 */
  double theta_wd;        /* Definition 2 threshold: 0.9 */
  double theta_wc;        /* Definition 1 threshold: 1e-2 */
  double sigma_wc;        /* switch criterion of Section 3.6: 0.5 */
  double inner_tol;       /* option #3 accuracy (PCTL p_alpha): 1e-2 */
  int inner_maxit;        /* option #3 cycle cap: 100 */
  int nvcyc_group, nvcyc_E, nvcyc_I, nvcyc_other; /* option #2 cycles per inverse */
  int jacobi_sweeps;      /* option #1 sweeps: 1 */
  int adaptive;           /* 1: Section 3.6 coupling drops + Section 3.5 option #1/#2 choice */
  uint64_t seed;          /* PMIS weight seed */
  int inner_mode;         /* 1: option #3 (V-cycles to inner_tol) for the inverses Section 4 names:
                             C_E, C_g (Schur1), S_g, S_I (Schur2), the block relaxations of PCTL */
  int interp_type;        /* 0: classical modified (Section 3.1); 1: extended+i (distance two) */
  int smoother;           /* 0: l1-Jacobi; 1: Gauss-Seidel in C/F order (Section 3.1's hybrid GS), read
                             as multicolour GS: C colours then F colours on the way down, the reverse up */
  int agg_levels;         /* levels, from the finest, coarsened aggressively (Section 3.1): a second PMIS
                             pass on the Galerkin operator of the first, which is not kept as a level;
                             P = P1 P2 (two-stage interpolation).  0: none (default) */
  int opt4_steps;         /* option #4 (Section 3.5), 0: off.  K > 0: the Schur complement whose inner
                             inverse is one block -- S_I = A_I - D_IE A_E^{-1} D_EI (Schur2) and
                             C_E = A_E - D_EI A_I^{-1} D_IE (Schur1) -- is inverted by K steps of
                             w^(0) = 0, w^(k+1) = A_a^{-1}(q + D_ab A_b^{-1} D_ba w^(k)), with A_a^{-1},
                             A_b^{-1} by option #1/#2 (or #3 under inner_mode); forward apply only */
} or_opts;

/* preconditioner kinds */
enum { OR_AMG = 0, OR_PCTL = 1, OR_SCHUR1 = 2, OR_SCHUR2 = 3, OR_BD = 4, OR_BLT = 5 };

/* operator ids handed to an inverse callback: id = kind*64 + component */
enum { OP_A = 0, OP_CE = 1, OP_CG = 2, OP_SG = 3, OP_SI = 4, OP_AC = 5, OP_MONO = 6 };

typedef void (*or_inv_cb)(void *ctx, int op, int comp, int N, const double *rhs, double *out);

void or_default_opts(or_opts *o);

/* i-th output (0-based) of a splitmix64 generator whose state starts at state0 */
uint64_t or_splitmix64(uint64_t state0, uint64_t i);
/* counter-based splitmix64 uniform in [0,1): same definition as the input module */
double or_uniform(uint64_t seed, uint64_t stream, uint64_t i);

/* CSR handles */
or_csr *or_csr_new(int n, int m, int nnz, const int *rp, const int *ci, const double *v);
void or_csr_info(const or_csr *A, int *n, int *m, int *nnz);
void or_csr_export(const or_csr *A, int *rp, int *ci, double *v);
void or_csr_free(or_csr *A);
void or_spmv(const or_csr *A, const double *x, double *y);
or_csr *or_transpose(const or_csr *A);
or_csr *or_spgemm(const or_csr *X, const or_csr *Y);

/* AMG setup building blocks (Section 3.1) */
void or_strength(const or_csr *A, double theta, uint8_t *S);
int or_pmis(const or_csr *A, const uint8_t *S, uint64_t seed, int level, int8_t *CF);
/* Colouring of the symmetrised graph of A (i ~ j when a_ij or a_ji is stored)
   by Jones-Plassmann rounds with weights u_i = or_uniform(seed, 2000 + level, i): each round every
   uncoloured point whose weight beats all uncoloured neighbours (ties: larger
   index) takes the smallest colour no coloured neighbour has.  Returns the
   number of colours. */
int or_colour(const or_csr *A, uint64_t seed, int level, int *colour);
/* same rounds with caller-given weights (ties broken by the larger index) */
int or_pmis_weights(const or_csr *A, const uint8_t *S, const double *w, int8_t *CF);
or_csr *or_interp(const or_csr *A, const uint8_t *S, const int8_t *CF);
/* extended+i (distance-two) interpolation, De Sterck, Falgout, Nolting, Yang 2008 */
or_csr *or_interp_exti(const or_csr *A, const uint8_t *S, const int8_t *CF);
or_csr *or_rap(const or_csr *A, const or_csr *P);

/* AMG hierarchy */
typedef struct or_amg or_amg;
or_amg *or_amg_setup(const or_csr *A, const or_opts *o);
int or_amg_nlevels(const or_amg *h);
const or_csr *or_amg_A(const or_amg *h, int l);
const or_csr *or_amg_P(const or_amg *h, int l);
const int8_t *or_amg_CF(const or_amg *h, int l);
/* Gauss-Seidel sweep index of each point of level l (smoother 1; NULL otherwise
   and on the coarsest level): C points by colour, then F points by colour,
   empty classes skipped; *nkeys = number of sweeps */
const int *or_amg_key(const or_amg *h, int l, int *nkeys);
int or_amg_coarse_is_lu(const or_amg *h);
void or_vcycle(const or_amg *h, const double *b, double *x);
void or_vcycle_T(const or_amg *h, const double *b, double *x);
void or_amg_free(or_amg *h);

/* dense LU with partial pivoting (coarsest level) */
int or_lu_factor(int n, double *a, int *piv);
void or_lu_solve(int n, const double *lu, const int *piv, const double *b, double *x);
void or_lu_solve_T(int n, const double *lu, const int *piv, const double *b, double *x);

/* indicators (Definitions 1 and 2) */
double or_gamma_wd(const or_csr *A, double theta_wd);
double or_gamma_wc(int N, const double *d_ab, const double *diag_a, double theta_wc);

/* block preconditioner on the monolithic block-major matrix */
typedef struct or_block or_block;
or_block *or_block_setup(const or_csr *A, int G, int N, int kind, const or_opts *o);
void or_block_apply(or_block *B, const double *v, double *z, or_inv_cb cb, void *ctx);
void or_block_apply_T(or_block *B, const double *v, double *z);
int or_block_ninv(const or_block *B);
int or_block_nmatvec(const or_block *B);
int or_block_dropped(const or_block *B, int a, int b);
int or_block_use_jacobi(const or_block *B, int op, int comp);
long or_block_cycles(const or_block *B, int op, int comp); /* V-cycles spent by one inverse */
const or_amg *or_block_amg(const or_block *B, int op, int comp);
const double *or_block_vec(const or_block *B, int which, int comp); /* 0: p_alpha, 1: diag of op */
const or_csr *or_block_Ac(const or_block *B);
void or_block_free(or_block *B);

/* right-preconditioned FGMRES(m), Section 2 / 4; M == NULL means identity.
   Returns 0 converged, 1 iteration cap, 2 Arnoldi breakdown that left the
   tolerance unmet (or a singular least-squares problem: x unchanged),
   3 non-finite residual. */
int or_fgmres(const or_csr *A, or_block *M, int transpose, const double *b, double *x,
              double tol, int restart, int maxit, int *iters, double *relres, double *hist);

/* adjoint gradient over A's pattern: g_k = -lambda[row(k)] * x[col(k)] */
void or_grad_vals(const or_csr *A, const double *x, const double *lambda, double *g);

#ifdef __cplusplus
}
#endif
#endif
