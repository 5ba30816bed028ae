/*
 * mgd_oracle.c -- FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see the header).
 *
 * Built with -O2 -ffp-contract=off so that every product and sum is rounded
 * exactly as written.  Plain loops, no blocking, no reordering.
 *
 * Method (Yue, Zhang, Xu, Shu, Shi, "Algebraic multigrid block preconditioning
 * for multi-group radiation diffusion equations"):
 *   Section 3.1  monolithic classical AMG (strength 0.25, V(1,1), classical
 *                modified interpolation, Galerkin coarse operators, <=100
 *                coarsest unknowns solved by Gaussian elimination)
 *   Section 3.3  PCTL two-level preconditioner, Eq. 3.3
 *   Section 3.4  Schur1 (Eq. 3.1 and its five-stage apply), Schur2 (Eq. 3.2
 *                and its three-stage apply)
 *   Section 3.5  options #1-#3 for approximate inverses, Definition 2
 *   Section 3.6  adaptive coupling drops, Definition 1, Remarks (BLT / BD)
 *   Section 4    GMRES(30) stopping rule on the relative residual
 *
 * Readings where the paper is silent or names a method it does not define:
 *   - coarsening is PMIS (De Sterck, Yang, Heys 2006) with seeded weights
 *     w_i = |S^T_i| + u_i instead of Falgout coarsening;
 *   - smoothing is l1-Jacobi (Baker, Falgout, Kolev, Yang 2011) with weight 1
 *     and D_ii = sum_j |a_ij| instead of hybrid Gauss-Seidel;
 *   - no aggressive coarsening, no interpolation truncation, no row-sum cutoff;
 *   - a level whose coarsening stalls (no C point, or all C) with more than
 *     max_coarse unknowns becomes the coarsest level and is relaxed by two
 *     l1-Jacobi sweeps;
 *   - the Krylov method is flexible GMRES (right preconditioning), restart 30.
 */
#include "mgd_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL
#define STREAM_PMIS 1000ULL

static void *xmalloc(size_t sz) {
  void *p = malloc(sz ? sz : 1);
  if (!p) {
    fprintf(stderr, "oracle: out of memory (%zu bytes)\n", sz);
    abort();
  }
  return p;
}
static void *xcalloc(size_t n, size_t sz) {
  void *p = calloc(n ? n : 1, sz ? sz : 1);
  if (!p) {
    fprintf(stderr, "oracle: out of memory\n");
    abort();
  }
  return p;
}

/* ------------------------------------------------------------------ */
/* splitmix64 counter generator (Steele, Lea, Flood 2014)               */
/* ------------------------------------------------------------------ */
static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t or_splitmix64(uint64_t state0, uint64_t i) { return mix64(state0 + (i + 1) * GOLDEN); }

double or_uniform(uint64_t seed, uint64_t stream, uint64_t i) {
  uint64_t key = mix64(mix64(seed + GOLDEN) + stream * GOLDEN);
  uint64_t z = mix64(key + (i + 1) * GOLDEN);
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

void or_default_opts(or_opts *o) {
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
  o->inner_mode = 0;
  o->interp_type = 0;
  o->smoother = 0;
  o->agg_levels = 0;
  o->opt4_steps = 0;
}

/* ------------------------------------------------------------------ */
/* CSR utilities                                                        */
/* ------------------------------------------------------------------ */
static or_csr *csr_alloc(int n, int m, int nnz) {
  or_csr *A = (or_csr *)xmalloc(sizeof(or_csr));
  A->n = n;
  A->m = m;
  A->nnz = nnz;
  A->rp = (int *)xcalloc((size_t)n + 1, sizeof(int));
  A->ci = (int *)xmalloc((size_t)nnz * sizeof(int));
  A->v = (double *)xmalloc((size_t)nnz * sizeof(double));
  return A;
}

or_csr *or_csr_new(int n, int m, int nnz, const int *rp, const int *ci, const double *v) {
  or_csr *A = csr_alloc(n, m, nnz);
  memcpy(A->rp, rp, ((size_t)n + 1) * sizeof(int));
  memcpy(A->ci, ci, (size_t)nnz * sizeof(int));
  memcpy(A->v, v, (size_t)nnz * sizeof(double));
  return A;
}

static or_csr *csr_copy(const or_csr *A) { return or_csr_new(A->n, A->m, A->nnz, A->rp, A->ci, A->v); }

void or_csr_info(const or_csr *A, int *n, int *m, int *nnz) {
  *n = A->n;
  *m = A->m;
  *nnz = A->nnz;
}

void or_csr_export(const or_csr *A, int *rp, int *ci, double *v) {
  if (rp) memcpy(rp, A->rp, ((size_t)A->n + 1) * sizeof(int));
  if (ci) memcpy(ci, A->ci, (size_t)A->nnz * sizeof(int));
  if (v) memcpy(v, A->v, (size_t)A->nnz * sizeof(double));
}

void or_csr_free(or_csr *A) {
  if (!A) return;
  free(A->rp);
  free(A->ci);
  free(A->v);
  free(A);
}

/* y = A x, each row summed left to right in stored column order */
void or_spmv(const or_csr *A, const double *x, double *y) {
  for (int i = 0; i < A->n; ++i) {
    double s = 0.0;
    for (int p = A->rp[i]; p < A->rp[i + 1]; ++p) s += A->v[p] * x[A->ci[p]];
    y[i] = s;
  }
}

/* r = b - A x */
static void residual(const or_csr *A, const double *b, const double *x, double *r) {
  for (int i = 0; i < A->n; ++i) {
    double s = 0.0;
    for (int p = A->rp[i]; p < A->rp[i + 1]; ++p) s += A->v[p] * x[A->ci[p]];
    r[i] = b[i] - s;
  }
}

/* explicit transpose; rows of the result come out with sorted columns
   because the source rows are scanned in increasing order */
or_csr *or_transpose(const or_csr *A) {
  or_csr *T = csr_alloc(A->m, A->n, A->nnz);
  for (int p = 0; p < A->nnz; ++p) T->rp[A->ci[p] + 1]++;
  for (int j = 0; j < A->m; ++j) T->rp[j + 1] += T->rp[j];
  int *next = (int *)xmalloc((size_t)A->m * sizeof(int));
  memcpy(next, T->rp, (size_t)A->m * sizeof(int));
  for (int i = 0; i < A->n; ++i)
    for (int p = A->rp[i]; p < A->rp[i + 1]; ++p) {
      int q = next[A->ci[p]]++;
      T->ci[q] = i;
      T->v[q] = A->v[p];
    }
  free(next);
  return T;
}

/* sort (col, val) pairs of one row by column (insertion sort: rows are short) */
static void sort_row(int *c, double *v, int len) {
  for (int a = 1; a < len; ++a) {
    int cc = c[a];
    double vv = v[a];
    int b = a - 1;
    while (b >= 0 && c[b] > cc) {
      c[b + 1] = c[b];
      v[b + 1] = v[b];
      --b;
    }
    c[b + 1] = cc;
    v[b + 1] = vv;
  }
}

/* C = X Y, row by row (Gustavson).  For an output entry (i, j) the products
   x_ik y_kj are accumulated in the order of k along row i of X; the first
   product initialises the entry.  Entries that cancel to zero are kept. */
or_csr *or_spgemm(const or_csr *X, const or_csr *Y) {
  int n = X->n, m = Y->m;
  int *marker = (int *)xmalloc((size_t)m * sizeof(int));
  for (int j = 0; j < m; ++j) marker[j] = -1;
  int *cnt = (int *)xcalloc((size_t)n + 1, sizeof(int));
  for (int i = 0; i < n; ++i) {
    int c = 0;
    for (int p = X->rp[i]; p < X->rp[i + 1]; ++p) {
      int k = X->ci[p];
      for (int q = Y->rp[k]; q < Y->rp[k + 1]; ++q) {
        int j = Y->ci[q];
        if (marker[j] != i) {
          marker[j] = i;
          ++c;
        }
      }
    }
    cnt[i + 1] = c;
  }
  for (int i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
  or_csr *C = csr_alloc(n, m, cnt[n]);
  memcpy(C->rp, cnt, ((size_t)n + 1) * sizeof(int));
  free(cnt);
  int *slot = (int *)xmalloc((size_t)m * sizeof(int));
  for (int j = 0; j < m; ++j) marker[j] = -1;
  for (int i = 0; i < n; ++i) {
    int base = C->rp[i], len = 0;
    for (int p = X->rp[i]; p < X->rp[i + 1]; ++p) {
      int k = X->ci[p];
      double xv = X->v[p];
      for (int q = Y->rp[k]; q < Y->rp[k + 1]; ++q) {
        int j = Y->ci[q];
        double prod = xv * Y->v[q];
        if (marker[j] != i) {
          marker[j] = i;
          slot[j] = base + len;
          C->ci[base + len] = j;
          C->v[base + len] = prod;
          ++len;
        } else {
          C->v[slot[j]] = C->v[slot[j]] + prod;
        }
      }
    }
    sort_row(C->ci + base, C->v + base, len);
  }
  free(marker);
  free(slot);
  return C;
}

/* ------------------------------------------------------------------ */
/* Strength of connection, Section 3.1 (threshold 0.25):               */
/*   j is a strong connection of i if i != j and                        */
/*   -a_ij >= theta * max_{k != i} (-a_ik), with that maximum > 0.      */
/* ------------------------------------------------------------------ */
void or_strength(const or_csr *A, double theta, uint8_t *S) {
  for (int i = 0; i < A->n; ++i) {
    double mx = 0.0;
    for (int p = A->rp[i]; p < A->rp[i + 1]; ++p)
      if (A->ci[p] != i && -A->v[p] > mx) mx = -A->v[p];
    double thr = theta * mx;
    for (int p = A->rp[i]; p < A->rp[i + 1]; ++p)
      S[p] = (uint8_t)(A->ci[p] != i && mx > 0.0 && -A->v[p] >= thr);
  }
}

/* ------------------------------------------------------------------ */
/* PMIS C/F splitting (De Sterck, Yang, Heys 2006), seeded weights.     */
/*   CF: 1 = C, -1 = F.  Returns the number of C points.                */
/* ------------------------------------------------------------------ */
static int pmis_beats(const double *w, int i, int j) {
  return w[i] > w[j] || (w[i] == w[j] && i > j);
}

static int pmis_core(const or_csr *A, const uint8_t *S, const double *wext, uint64_t seed, int level, int8_t *CF) {
  int n = A->n;
  /* S^T: for every point i, the points that strongly depend on i */
  int *trp = (int *)xcalloc((size_t)n + 1, sizeof(int));
  for (int i = 0; i < n; ++i)
    for (int p = A->rp[i]; p < A->rp[i + 1]; ++p)
      if (S[p]) trp[A->ci[p] + 1]++;
  for (int i = 0; i < n; ++i) trp[i + 1] += trp[i];
  int *tci = (int *)xmalloc((size_t)trp[n] * sizeof(int) + 4);
  int *next = (int *)xmalloc((size_t)n * sizeof(int) + 4);
  memcpy(next, trp, (size_t)n * sizeof(int));
  for (int i = 0; i < n; ++i)
    for (int p = A->rp[i]; p < A->rp[i + 1]; ++p)
      if (S[p]) tci[next[A->ci[p]]++] = i;
  free(next);

  double *w = (double *)xmalloc((size_t)n * sizeof(double) + 8);
  for (int i = 0; i < n; ++i)
    w[i] = wext ? wext[i]
                : (double)(trp[i + 1] - trp[i]) + or_uniform(seed, STREAM_PMIS + (uint64_t)level, (uint64_t)i);

  /* initial decisions: isolated points and points nobody depends on are F */
  for (int i = 0; i < n; ++i) {
    int ns = 0;
    for (int p = A->rp[i]; p < A->rp[i + 1]; ++p) ns += S[p];
    int nst = trp[i + 1] - trp[i];
    if (ns == 0 && nst == 0)
      CF[i] = -1;
    else if (w[i] < 1.0)
      CF[i] = -1;
    else
      CF[i] = 0;
  }
  uint8_t *newc = (uint8_t *)xcalloc((size_t)n, 1);
  for (;;) {
    int undecided = 0;
    for (int i = 0; i < n; ++i) undecided += (CF[i] == 0);
    if (!undecided) break;
    /* C: local maxima among undecided neighbours in S_i and S^T_i */
    for (int i = 0; i < n; ++i) {
      newc[i] = 0;
      if (CF[i] != 0) continue;
      int ismax = 1;
      for (int p = A->rp[i]; p < A->rp[i + 1] && ismax; ++p)
        if (S[p] && CF[A->ci[p]] == 0 && !pmis_beats(w, i, A->ci[p])) ismax = 0;
      for (int p = trp[i]; p < trp[i + 1] && ismax; ++p)
        if (CF[tci[p]] == 0 && !pmis_beats(w, i, tci[p])) ismax = 0;
      newc[i] = (uint8_t)ismax;
    }
    for (int i = 0; i < n; ++i)
      if (newc[i]) CF[i] = 1;
    /* F: undecided points that strongly depend on a C point */
    for (int i = 0; i < n; ++i) {
      if (CF[i] != 0) continue;
      for (int p = A->rp[i]; p < A->rp[i + 1]; ++p)
        if (S[p] && CF[A->ci[p]] == 1) {
          CF[i] = -1;
          break;
        }
    }
  }
  int nc = 0;
  for (int i = 0; i < n; ++i) nc += (CF[i] == 1);
  free(newc);
  free(w);
  free(trp);
  free(tci);
  return nc;
}

int or_pmis(const or_csr *A, const uint8_t *S, uint64_t seed, int level, int8_t *CF) {
  return pmis_core(A, S, NULL, seed, level, CF);
}

int or_pmis_weights(const or_csr *A, const uint8_t *S, const double *w, int8_t *CF) {
  return pmis_core(A, S, w, 0, 0, CF);
}

/* Jones-Plassmann colouring (the Gauss-Seidel order of the smoother) of the
   symmetrised graph: i and j are neighbours when a_ij or a_ji is stored.
   Rounds over the uncoloured points, all taken simultaneously from the
   colours of the previous round. */
static int colour_taken(const or_csr *A, const or_csr *AT, int i, const int *colour, int c) {
  for (int p = A->rp[i]; p < A->rp[i + 1]; ++p)
    if (A->ci[p] != i && colour[A->ci[p]] == c) return 1;
  for (int p = AT->rp[i]; p < AT->rp[i + 1]; ++p)
    if (AT->ci[p] != i && colour[AT->ci[p]] == c) return 1;
  return 0;
}

static int colour_beaten(const or_csr *M, int i, const int *colour, const double *w) {
  for (int p = M->rp[i]; p < M->rp[i + 1]; ++p) {
    int j = M->ci[p];
    if (j == i || colour[j] >= 0) continue;
    if (w[j] > w[i] || (w[j] == w[i] && j > i)) return 1;
  }
  return 0;
}

int or_colour(const or_csr *A, uint64_t seed, int level, int *colour) {
  int n = A->n;
  or_csr *AT = or_transpose(A);
  double *w = (double *)xmalloc((size_t)n * sizeof(double) + 8);
  int *next = (int *)xmalloc((size_t)n * sizeof(int) + 8);
  for (int i = 0; i < n; ++i) {
    w[i] = or_uniform(seed, 2000ULL + (uint64_t)level, (uint64_t)i);
    colour[i] = -1;
  }
  int left = n, ncol = 0;
  while (left > 0) {
    for (int i = 0; i < n; ++i) {
      next[i] = colour[i];
      if (colour[i] >= 0) continue;
      if (colour_beaten(A, i, colour, w) || colour_beaten(AT, i, colour, w)) continue;
      int c = 0;  /* the smallest colour that no coloured neighbour has */
      while (colour_taken(A, AT, i, colour, c)) ++c;
      next[i] = c;
    }
    left = 0;
    for (int i = 0; i < n; ++i) {
      colour[i] = next[i];
      if (colour[i] < 0) ++left;
      else if (colour[i] + 1 > ncol) ncol = colour[i] + 1;
    }
  }
  or_csr_free(AT);
  free(w);
  free(next);
  return ncol;
}

/* ------------------------------------------------------------------ */
/* Classical modified interpolation (Ruge-Stueben), Section 3.1.        */
/* For an F point i with strong C neighbours C_i, strong F neighbours   */
/* F_i and the remaining neighbours W_i (weak ones, and strong F        */
/* neighbours with no opposite-sign connection into C_i):               */
/*   w_ij = -( a_ij + sum_{k in F_i} a_ik abar_kj / sum_{m in C_i}      */
/*             abar_km ) / ( a_ii + sum_{n in W_i} a_in ),  j in C_i,   */
/* with abar_km = a_km when its sign differs from a_kk, else 0.         */
/* C points interpolate by injection.  F points without C neighbours    */
/* get an empty row.  Sums run in the row's stored column order.        */
/* ------------------------------------------------------------------ */
static int opposite_sign(double akm, double akk) { return akk > 0.0 ? (akm < 0.0) : (akm > 0.0); }

or_csr *or_interp(const or_csr *A, const uint8_t *S, const int8_t *CF) {
  int n = A->n;
  int *cidx = (int *)xmalloc((size_t)n * sizeof(int) + 4);
  int nc = 0;
  for (int i = 0; i < n; ++i) cidx[i] = (CF[i] == 1) ? nc++ : -1;
  int *rp = (int *)xcalloc((size_t)n + 1, sizeof(int));
  for (int i = 0; i < n; ++i) {
    int c = 0;
    if (CF[i] == 1)
      c = 1;
    else
      for (int p = A->rp[i]; p < A->rp[i + 1]; ++p)
        if (S[p] && CF[A->ci[p]] == 1) ++c;
    rp[i + 1] = c;
  }
  for (int i = 0; i < n; ++i) rp[i + 1] += rp[i];
  or_csr *P = csr_alloc(n, nc, rp[n]);
  memcpy(P->rp, rp, ((size_t)n + 1) * sizeof(int));
  free(rp);

  for (int i = 0; i < n; ++i) {
    int base = P->rp[i];
    if (CF[i] == 1) {
      P->ci[base] = cidx[i];
      P->v[base] = 1.0;
      continue;
    }
    int len = P->rp[i + 1] - base;
    if (len == 0) continue;
    /* numerators start from the direct terms a_ij, j in C_i (row order) */
    int t = 0;
    double diag = 0.0;
    for (int p = A->rp[i]; p < A->rp[i + 1]; ++p) {
      int j = A->ci[p];
      if (j == i) diag = A->v[p];
      if (S[p] && CF[j] == 1) {
        P->ci[base + t] = j; /* fine index for now */
        P->v[base + t] = A->v[p];
        ++t;
      }
    }
    for (int p = A->rp[i]; p < A->rp[i + 1]; ++p) {
      int k = A->ci[p];
      if (k == i) continue;
      double aik = A->v[p];
      if (S[p] && CF[k] == 1) continue;
      if (S[p] && CF[k] == -1) {
        double akk = 0.0;
        for (int q = A->rp[k]; q < A->rp[k + 1]; ++q)
          if (A->ci[q] == k) akk = A->v[q];
        double denom = 0.0;
        for (int q = A->rp[k]; q < A->rp[k + 1]; ++q) {
          int m = A->ci[q];
          for (int s = 0; s < len; ++s)
            if (P->ci[base + s] == m) {
              if (opposite_sign(A->v[q], akk)) denom = denom + A->v[q];
              break;
            }
        }
        if (denom == 0.0) {
          diag = diag + aik;
        } else {
          for (int q = A->rp[k]; q < A->rp[k + 1]; ++q) {
            int m = A->ci[q];
            for (int s = 0; s < len; ++s)
              if (P->ci[base + s] == m) {
                if (opposite_sign(A->v[q], akk)) {
                  double prod = aik * A->v[q];
                  P->v[base + s] = P->v[base + s] + prod / denom;
                }
                break;
              }
          }
        }
      } else {
        diag = diag + aik; /* weak neighbour */
      }
    }
    for (int s = 0; s < len; ++s) {
      P->v[base + s] = (diag != 0.0) ? -P->v[base + s] / diag : 0.0;
      P->ci[base + s] = cidx[P->ci[base + s]];
    }
  }
  free(cidx);
  return P;
}

/* ------------------------------------------------------------------ */
/* Extended+i interpolation (De Sterck, Falgout, Nolting, Yang, "Distance-two */
/* interpolation for parallel algebraic multigrid", NLAA 2008).  For an F   */
/* point i the interpolatory set is C^_i = (strong C neighbours of i) united */
/* with the strong C neighbours of i's strong F neighbours, and             */
/*   w_ij = -( a_ij + sum_{k in F_i} a_ik abar_kj / d_k ) / a~_ii,          */
/*   a~_ii = a_ii + sum_{n weak, not in C^_i} a_in                          */
/*                + sum_{k in F_i} a_ik abar_ki / d_k,                      */
/*   d_k = sum_{l in C^_i or l = i} abar_kl,                                */
/* abar as in the classical formula; a_ij = 0 for j not adjacent to i.  A   */
/* strong F neighbour with d_k = 0 is lumped into the diagonal.  C^_i is    */
/* built in the order: strong C neighbours of i (row order), then for each  */
/* strong F neighbour k (row order) its strong C neighbours (row order) not */
/* yet listed; sums run in row i's stored order, then row k's.              */
/* ------------------------------------------------------------------ */
static int in_list(const int *list, int len, int j) {
  for (int s = 0; s < len; ++s)
    if (list[s] == j) return s;
  return -1;
}

or_csr *or_interp_exti(const or_csr *A, const uint8_t *S, const int8_t *CF) {
  int n = A->n;
  int *cidx = (int *)xmalloc((size_t)n * sizeof(int) + 4);
  int nc = 0;
  for (int i = 0; i < n; ++i) cidx[i] = (CF[i] == 1) ? nc++ : -1;
  /* pass 1: interpolatory sets and their sizes */
  int *rp = (int *)xcalloc((size_t)n + 1, sizeof(int));
  int cap = 64;
  int *list = (int *)xmalloc((size_t)cap * sizeof(int));
  for (int i = 0; i < n; ++i) {
    int len = 0;
    if (CF[i] == 1) {
      rp[i + 1] = 1;
      continue;
    }
    for (int p = A->rp[i]; p < A->rp[i + 1]; ++p) {
      int j = A->ci[p];
      if (S[p] && CF[j] == 1 && in_list(list, len, j) < 0) {
        if (len == cap) list = (int *)realloc(list, (size_t)(cap *= 2) * sizeof(int));
        list[len++] = j;
      }
    }
    for (int p = A->rp[i]; p < A->rp[i + 1]; ++p) {
      int k = A->ci[p];
      if (!(S[p] && CF[k] == -1)) continue;
      for (int q = A->rp[k]; q < A->rp[k + 1]; ++q) {
        int m = A->ci[q];
        if (S[q] && CF[m] == 1 && in_list(list, len, m) < 0) {
          if (len == cap) list = (int *)realloc(list, (size_t)(cap *= 2) * sizeof(int));
          list[len++] = m;
        }
      }
    }
    rp[i + 1] = len;
  }
  for (int i = 0; i < n; ++i) rp[i + 1] += rp[i];
  or_csr *P = csr_alloc(n, nc, rp[n]);
  memcpy(P->rp, rp, ((size_t)n + 1) * sizeof(int));
  free(rp);
  /* pass 2: weights */
  for (int i = 0; i < n; ++i) {
    int base = P->rp[i], len = P->rp[i + 1] - base;
    if (CF[i] == 1) {
      P->ci[base] = cidx[i];
      P->v[base] = 1.0;
      continue;
    }
    if (len == 0) continue;
    int *L = P->ci + base;  /* fine indices while building */
    double *num = P->v + base;
    int t = 0;
    for (int p = A->rp[i]; p < A->rp[i + 1]; ++p) {
      int j = A->ci[p];
      if (S[p] && CF[j] == 1 && in_list(L, t, j) < 0) L[t++] = j;
    }
    for (int p = A->rp[i]; p < A->rp[i + 1]; ++p) {
      int k = A->ci[p];
      if (!(S[p] && CF[k] == -1)) continue;
      for (int q = A->rp[k]; q < A->rp[k + 1]; ++q) {
        int m = A->ci[q];
        if (S[q] && CF[m] == 1 && in_list(L, t, m) < 0) L[t++] = m;
      }
    }
    for (int s2 = 0; s2 < len; ++s2) num[s2] = 0.0;
    double diag = 0.0;
    for (int p = A->rp[i]; p < A->rp[i + 1]; ++p) {
      int j = A->ci[p];
      if (j == i) {
        diag = A->v[p];
        continue;
      }
      int sj = in_list(L, len, j);
      if (sj >= 0) num[sj] = A->v[p]; /* a_ij for neighbours in C^_i */
    }
    for (int p = A->rp[i]; p < A->rp[i + 1]; ++p) {
      int k = A->ci[p];
      if (k == i) continue;
      double aik = A->v[p];
      if (S[p] && CF[k] == 1) continue;
      if (S[p] && CF[k] == -1) {
        double akk = 0.0;
        for (int q = A->rp[k]; q < A->rp[k + 1]; ++q)
          if (A->ci[q] == k) akk = A->v[q];
        double denom = 0.0;
        for (int q = A->rp[k]; q < A->rp[k + 1]; ++q) {
          int l = A->ci[q];
          if ((l == i || in_list(L, len, l) >= 0) && opposite_sign(A->v[q], akk)) denom = denom + A->v[q];
        }
        if (denom == 0.0) {
          diag = diag + aik;
        } else {
          for (int q = A->rp[k]; q < A->rp[k + 1]; ++q) {
            int l = A->ci[q];
            if (!opposite_sign(A->v[q], akk)) continue;
            double prod = aik * A->v[q];
            if (l == i) {
              diag = diag + prod / denom;
            } else {
              int sl = in_list(L, len, l);
              if (sl >= 0) num[sl] = num[sl] + prod / denom;
            }
          }
        }
      } else if (in_list(L, len, k) < 0) {
        diag = diag + aik; /* weak neighbour outside C^_i */
      }
    }
    /* finalise and sort the row by coarse index */
    for (int s2 = 0; s2 < len; ++s2) {
      num[s2] = (diag != 0.0) ? -num[s2] / diag : 0.0;
      L[s2] = cidx[L[s2]];
    }
    sort_row(L, num, len);
  }
  free(list);
  free(cidx);
  return P;
}

/* Galerkin coarse operator A_c = R A P with R = P^T (AP first) */
or_csr *or_rap(const or_csr *A, const or_csr *P) {
  or_csr *AP = or_spgemm(A, P);
  or_csr *R = or_transpose(P);
  or_csr *Ac = or_spgemm(R, AP);
  or_csr_free(AP);
  or_csr_free(R);
  return Ac;
}

/* ------------------------------------------------------------------ */
/* Dense LU with partial pivoting (coarsest level, Section 3.1)         */
/* a: row-major n x n, overwritten by L (unit, below) and U            */
/* ------------------------------------------------------------------ */
int or_lu_factor(int n, double *a, int *piv) {
  for (int k = 0; k < n; ++k) {
    int pr = k;
    double best = fabs(a[(size_t)k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (fabs(a[(size_t)i * n + k]) > best) {
        best = fabs(a[(size_t)i * n + k]);
        pr = i;
      }
    piv[k] = pr;
    if (best == 0.0) return -1;
    if (pr != k)
      for (int j = 0; j < n; ++j) {
        double t = a[(size_t)k * n + j];
        a[(size_t)k * n + j] = a[(size_t)pr * n + j];
        a[(size_t)pr * n + j] = t;
      }
    for (int i = k + 1; i < n; ++i) {
      double l = a[(size_t)i * n + k] / a[(size_t)k * n + k];
      a[(size_t)i * n + k] = l;
      for (int j = k + 1; j < n; ++j) a[(size_t)i * n + j] -= l * a[(size_t)k * n + j];
    }
  }
  return 0;
}

void or_lu_solve(int n, const double *lu, const int *piv, const double *b, double *x) {
  for (int i = 0; i < n; ++i) x[i] = b[i];
  for (int k = 0; k < n; ++k)
    if (piv[k] != k) {
      double t = x[k];
      x[k] = x[piv[k]];
      x[piv[k]] = t;
    }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) x[i] -= lu[(size_t)i * n + j] * x[j];
  for (int i = n - 1; i >= 0; --i) {
    for (int j = i + 1; j < n; ++j) x[i] -= lu[(size_t)i * n + j] * x[j];
    x[i] /= lu[(size_t)i * n + i];
  }
}

/* solve A^T x = b with A = P^T L U: U^T y = b, L^T z = y, x = P^T z */
void or_lu_solve_T(int n, const double *lu, const int *piv, const double *b, double *x) {
  for (int i = 0; i < n; ++i) x[i] = b[i];
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < i; ++j) x[i] -= lu[(size_t)j * n + i] * x[j];
    x[i] /= lu[(size_t)i * n + i];
  }
  for (int i = n - 1; i >= 0; --i)
    for (int j = i + 1; j < n; ++j) x[i] -= lu[(size_t)j * n + i] * x[j];
  for (int k = n - 1; k >= 0; --k)
    if (piv[k] != k) {
      double t = x[k];
      x[k] = x[piv[k]];
      x[piv[k]] = t;
    }
}

/* ------------------------------------------------------------------ */
/* AMG hierarchy and V(1,1) cycle                                       */
/* ------------------------------------------------------------------ */
struct or_amg {
  int L;              /* number of levels */
  or_csr **A, **P, **R, **AT;
  int8_t **CF;
  double **dinv;      /* inverse l1 row norms */
  double **w1, **w2, **w3; /* per-level work: x, b, r */
  int coarse_lu;      /* 1: dense LU at the coarsest level, 0: two l1-Jacobi sweeps */
  double *lu;
  int *piv;
  int smoother;       /* 0: l1-Jacobi; 1: Gauss-Seidel in C/F colour order */
  int **key;          /* smoother 1: sweep index per point (levels with a C/F split) */
  int *nkeys;
  double **gdinv;     /* smoother 1: 1 / a_ii */
};

static double *l1_dinv(const or_csr *A) {
  double *d = (double *)xmalloc((size_t)A->n * sizeof(double) + 8);
  for (int i = 0; i < A->n; ++i) {
    double s = 0.0;
    for (int p = A->rp[i]; p < A->rp[i + 1]; ++p) s += fabs(A->v[p]);
    d[i] = 1.0 / s;
  }
  return d;
}

/* Section 3.1's symmetric C/F relaxation order for level l: sweep keys
   C(colour 0), C(colour 1), ..., F(colour 0), F(colour 1), ..., with empty
   classes dropped; and the Gauss-Seidel diagonal 1 / a_ii */
static void gs_order(or_amg *h, int l, const or_csr *A, const int8_t *CF, uint64_t seed) {
  int n = A->n;
  int *col = (int *)xmalloc((size_t)n * sizeof(int) + 8);
  int ncol = or_colour(A, seed, l, col);
  int nraw = 2 * ncol;
  int *cnt = (int *)xcalloc((size_t)nraw + 1, sizeof(int));
  for (int i = 0; i < n; ++i) cnt[(CF[i] == 1 ? 0 : ncol) + col[i]]++;
  int *map = (int *)xmalloc((size_t)nraw * sizeof(int) + 8);
  int nk = 0;
  for (int k = 0; k < nraw; ++k) map[k] = cnt[k] > 0 ? nk++ : -1;
  h->key[l] = (int *)xmalloc((size_t)n * sizeof(int) + 8);
  for (int i = 0; i < n; ++i) h->key[l][i] = map[(CF[i] == 1 ? 0 : ncol) + col[i]];
  h->nkeys[l] = nk;
  h->gdinv[l] = (double *)xmalloc((size_t)n * sizeof(double) + 8);
  for (int i = 0; i < n; ++i) {
    double d = 1.0;
    for (int p = A->rp[i]; p < A->rp[i + 1]; ++p)
      if (A->ci[p] == i) d = A->v[p];
    h->gdinv[l][i] = 1.0 / d;
  }
  free(col);
  free(cnt);
  free(map);
}

/* Aggressive coarsening of level l (Section 3.1): the first pass gave CF and
   P1 = h->P[l].  A second strength + PMIS pass (weights from stream 1100 + l)
   on A1 = P1^T A P1 picks the final C points among the first pass's; P2
   interpolates from them to A1's points and P = P1 P2.  A1 is not a level.
   The level's C/F marks become: C where the first pass's C point stays C,
   F (-1) where it does not, the first pass's mark elsewhere.  If the second
   pass stalls (no C point, or all C) the level keeps the first pass. */
static void aggressive_pass(or_amg *h, int l, const or_csr *A, const or_opts *o) {
  or_csr *P1 = h->P[l];
  or_csr *A1 = or_rap(A, P1);
  int n1 = A1->n;
  uint8_t *S1 = (uint8_t *)xmalloc((size_t)A1->nnz + 1);
  or_strength(A1, o->theta_str, S1);
  int8_t *CF1 = (int8_t *)xmalloc((size_t)n1 + 1);
  int nc1 = or_pmis(A1, S1, o->seed, 100 + l, CF1);
  if (nc1 > 0 && nc1 < n1) {
    or_csr *P2 = o->interp_type == 1 ? or_interp_exti(A1, S1, CF1) : or_interp(A1, S1, CF1);
    h->P[l] = or_spgemm(P1, P2);
    int8_t *CF = h->CF[l];
    int c = 0;
    for (int i = 0; i < A->n; ++i) {
      if (CF[i] != 1) continue;
      CF[i] = CF1[c] == 1 ? 1 : -1;
      ++c;
    }
    or_csr_free(P1);
    or_csr_free(P2);
  }
  or_csr_free(A1);
  free(S1);
  free(CF1);
}

or_amg *or_amg_setup(const or_csr *A0, const or_opts *o) {
  int cap = o->max_levels > 0 ? o->max_levels : 1;
  or_amg *h = (or_amg *)xcalloc(1, sizeof(or_amg));
  h->A = (or_csr **)xcalloc((size_t)cap, sizeof(or_csr *));
  h->P = (or_csr **)xcalloc((size_t)cap, sizeof(or_csr *));
  h->R = (or_csr **)xcalloc((size_t)cap, sizeof(or_csr *));
  h->AT = (or_csr **)xcalloc((size_t)cap, sizeof(or_csr *));
  h->CF = (int8_t **)xcalloc((size_t)cap, sizeof(int8_t *));
  h->dinv = (double **)xcalloc((size_t)cap, sizeof(double *));
  h->w1 = (double **)xcalloc((size_t)cap, sizeof(double *));
  h->w2 = (double **)xcalloc((size_t)cap, sizeof(double *));
  h->w3 = (double **)xcalloc((size_t)cap, sizeof(double *));
  h->key = (int **)xcalloc((size_t)cap, sizeof(int *));
  h->nkeys = (int *)xcalloc((size_t)cap, sizeof(int));
  h->gdinv = (double **)xcalloc((size_t)cap, sizeof(double *));
  h->smoother = o->smoother;
  h->A[0] = csr_copy(A0);
  int l = 0;
  for (;;) {
    or_csr *A = h->A[l];
    h->dinv[l] = l1_dinv(A);
    h->w1[l] = (double *)xcalloc((size_t)A->n + 1, sizeof(double));
    h->w2[l] = (double *)xcalloc((size_t)A->n + 1, sizeof(double));
    h->w3[l] = (double *)xcalloc((size_t)A->n + 1, sizeof(double));
    if (A->n <= o->max_coarse || l == cap - 1) break;
    uint8_t *S = (uint8_t *)xmalloc((size_t)A->nnz + 1);
    or_strength(A, o->theta_str, S);
    int8_t *CF = (int8_t *)xmalloc((size_t)A->n + 1);
    int nc = or_pmis(A, S, o->seed, l, CF);
    if (nc == 0 || nc == A->n) {
      free(S);
      free(CF);
      break;
    }
    h->CF[l] = CF;
    h->P[l] = o->interp_type == 1 ? or_interp_exti(A, S, CF) : or_interp(A, S, CF);
    if (l < o->agg_levels) aggressive_pass(h, l, A, o);
    if (o->smoother == 1) gs_order(h, l, A, h->CF[l], o->seed);
    h->R[l] = or_transpose(h->P[l]);
    h->A[l + 1] = or_rap(A, h->P[l]);
    free(S);
    ++l;
  }
  h->L = l + 1;
  or_csr *Ac = h->A[l];
  if (Ac->n <= o->max_coarse) {
    int n = Ac->n;
    h->lu = (double *)xcalloc((size_t)n * n + 1, sizeof(double));
    h->piv = (int *)xcalloc((size_t)n + 1, sizeof(int));
    for (int i = 0; i < n; ++i)
      for (int p = Ac->rp[i]; p < Ac->rp[i + 1]; ++p) h->lu[(size_t)i * n + Ac->ci[p]] = Ac->v[p];
    h->coarse_lu = (or_lu_factor(n, h->lu, h->piv) == 0);
  }
  for (int k = 0; k < h->L; ++k) h->AT[k] = or_transpose(h->A[k]);
  return h;
}

int or_amg_nlevels(const or_amg *h) { return h->L; }
const or_csr *or_amg_A(const or_amg *h, int l) { return h->A[l]; }
const or_csr *or_amg_P(const or_amg *h, int l) { return l < h->L - 1 ? h->P[l] : NULL; }
const int8_t *or_amg_CF(const or_amg *h, int l) { return l < h->L - 1 ? h->CF[l] : NULL; }
int or_amg_coarse_is_lu(const or_amg *h) { return h->coarse_lu; }
const int *or_amg_key(const or_amg *h, int l, int *nkeys) {
  if (nkeys) *nkeys = (l < h->L - 1 && h->key[l]) ? h->nkeys[l] : 0;
  return l < h->L - 1 ? h->key[l] : NULL;
}

void or_amg_free(or_amg *h) {
  if (!h) return;
  for (int l = 0; l < h->L; ++l) {
    or_csr_free(h->A[l]);
    or_csr_free(h->P[l]);
    or_csr_free(h->R[l]);
    or_csr_free(h->AT[l]);
    free(h->CF[l]);
    free(h->dinv[l]);
    free(h->w1[l]);
    free(h->w2[l]);
    free(h->w3[l]);
    free(h->key[l]);
    free(h->gdinv[l]);
  }
  free(h->key);
  free(h->nkeys);
  free(h->gdinv);
  free(h->A);
  free(h->P);
  free(h->R);
  free(h->AT);
  free(h->CF);
  free(h->dinv);
  free(h->w1);
  free(h->w2);
  free(h->w3);
  free(h->lu);
  free(h->piv);
  free(h);
}

/* one Gauss-Seidel sweep over the points with sweep index k: no two of them
   are coupled (a colour class of the symmetrised graph), so each is updated
   from the current values of all other points: x_i += (b_i - sum_j a_ij x_j) / a_ii */
static void gs_sweep(const or_csr *A, const int *key, int k, const double *gdinv, const double *b, double *x) {
  for (int i = 0; i < A->n; ++i) {
    if (key[i] != k) continue;
    double s = 0.0;
    for (int p = A->rp[i]; p < A->rp[i + 1]; ++p) s += A->v[p] * x[A->ci[p]];
    x[i] = x[i] + (b[i] - s) * gdinv[i];
  }
}

/* one V(1,1) cycle with zero initial guess on level l.
   trans = 1 runs the adjoint cycle: same D, R and P, operators A_l^T and the
   transposed coarsest solve, which is the exact transpose of the cycle. */
static void vcycle_level(const or_amg *h, int l, int trans, const double *b, double *x) {
  const or_csr *A = trans ? h->AT[l] : h->A[l];
  const double *d = h->dinv[l];
  int n = A->n;
  if (l == h->L - 1) {
    if (h->coarse_lu) {
      if (trans)
        or_lu_solve_T(n, h->lu, h->piv, b, x);
      else
        or_lu_solve(n, h->lu, h->piv, b, x);
    } else {
      double *r = h->w3[l];
      for (int i = 0; i < n; ++i) x[i] = d[i] * b[i];
      residual(A, b, x, r);
      for (int i = 0; i < n; ++i) x[i] = x[i] + d[i] * r[i];
    }
    return;
  }
  double *r = h->w3[l];
  double *bc = h->w2[l + 1];
  double *xc = h->w1[l + 1];
  const or_csr *P = h->P[l], *R = h->R[l];
  if (h->smoother == 1) {
    /* down: Gauss-Seidel sweeps in key order (C points, then F points) from zero */
    for (int i = 0; i < n; ++i) x[i] = 0.0;
    for (int k = 0; k < h->nkeys[l]; ++k) gs_sweep(A, h->key[l], k, h->gdinv[l], b, x);
    residual(A, b, x, r);
    or_spmv(R, r, bc);
    vcycle_level(h, l + 1, trans, bc, xc);
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int p = P->rp[i]; p < P->rp[i + 1]; ++p) s += P->v[p] * xc[P->ci[p]];
      x[i] = x[i] + s;
    }
    /* up: the opposite traversal (F points, then C points) */
    for (int k = h->nkeys[l] - 1; k >= 0; --k) gs_sweep(A, h->key[l], k, h->gdinv[l], b, x);
    return;
  }
  for (int i = 0; i < n; ++i) x[i] = d[i] * b[i];     /* pre-smoothing from zero */
  residual(A, b, x, r);                               /* r = b - A x */
  or_spmv(R, r, bc);                                  /* restriction */
  vcycle_level(h, l + 1, trans, bc, xc);
  for (int i = 0; i < n; ++i) {                       /* prolongation */
    double s = 0.0;
    for (int p = P->rp[i]; p < P->rp[i + 1]; ++p) s += P->v[p] * xc[P->ci[p]];
    x[i] = x[i] + s;
  }
  residual(A, b, x, r);                               /* post-smoothing */
  for (int i = 0; i < n; ++i) x[i] = x[i] + d[i] * r[i];
}

void or_vcycle(const or_amg *h, const double *b, double *x) { vcycle_level(h, 0, 0, b, x); }
void or_vcycle_T(const or_amg *h, const double *b, double *x) { vcycle_level(h, 0, 1, b, x); }

/* ------------------------------------------------------------------ */
/* Indicators: Definition 2 (weak diagonal dominance) and Definition 1  */
/* (weak coupling)                                                      */
/* ------------------------------------------------------------------ */
double or_gamma_wd(const or_csr *A, double theta_wd) {
  int cnt = 0;
  for (int k = 0; k < A->n; ++k) {
    double rs = 0.0, akk = 0.0;
    for (int p = A->rp[k]; p < A->rp[k + 1]; ++p) {
      rs += A->v[p];
      if (A->ci[p] == k) akk = A->v[p];
    }
    if (rs < theta_wd * akk) ++cnt;
  }
  return A->n ? (double)cnt / (double)A->n : 0.0;
}

double or_gamma_wc(int N, const double *d_ab, const double *diag_a, double theta_wc) {
  int cnt = 0;
  for (int k = 0; k < N; ++k)
    if (-d_ab[k] <= theta_wc * diag_a[k]) ++cnt;
  return N ? (double)cnt / (double)N : 0.0;
}

/* ------------------------------------------------------------------ */
/* Block preconditioners (Sections 3.1, 3.3-3.6)                        */
/* component a: 0..G-1 groups, G = E, G+1 = I                           */
/* ------------------------------------------------------------------ */
typedef struct inv_t {
  or_csr *A;        /* operator being inverted (owned) */
  or_amg *amg;      /* option #2: its hierarchy */
  double *jdinv;    /* option #1: 1 / diag(A) */
  int use_jacobi;
  int accurate;     /* option #3: V-cycles until ||rhs - A x|| <= inner_tol ||rhs|| */
  int count;        /* sweeps (#1) or V-cycles (#2) */
  long cycles;      /* V-cycles spent by this inverse since setup */
} inv_t;

#define NOPS 7
struct or_block {
  int G, N, nc, kind;
  or_opts o;
  or_csr *Amono;
  or_csr **Ab;       /* diagonal blocks A_a */
  double **d;        /* d[a*nc+b]: coupling diagonal D_ab (NULL: absent or dropped) */
  int *dropped;
  double **diag;     /* diag(A_a) */
  inv_t *inv[NOPS];  /* inv[op][comp] */
  double **p;        /* PCTL p_a */
  or_csr *Ac;        /* PCTL coarse operator, Eq. 3.3 */
  int ninv, nmatvec; /* counts of the last apply (Table 1) */
  double *t1, *t2, *t3, *t4, *t5, *t6;
};

static int diag_pos(const or_csr *A, int i) {
  for (int p = A->rp[i]; p < A->rp[i + 1]; ++p)
    if (A->ci[p] == i) return p;
  return -1;
}

static void inv_build(or_block *B, int op, int comp, or_csr *A, int ncyc) {
  inv_t *iv = &B->inv[op][comp];
  iv->A = A;
  iv->use_jacobi = B->o.adaptive && or_gamma_wd(A, B->o.theta_wd) == 0.0;
  if (iv->use_jacobi) {
    iv->count = B->o.jacobi_sweeps;
    iv->jdinv = (double *)xmalloc((size_t)A->n * sizeof(double) + 8);
    for (int i = 0; i < A->n; ++i) {
      int p = diag_pos(A, i);
      iv->jdinv[i] = 1.0 / (p >= 0 ? A->v[p] : 1.0);
    }
  } else {
    iv->count = ncyc;
    iv->amg = or_amg_setup(A, &B->o);
    /* Section 4: inner accuracy 1e-2 for C_E, S_I, C_g, S_g and the PCTL block relaxations */
    iv->accurate = B->o.inner_mode &&
                   (op == OP_CE || op == OP_CG || op == OP_SG || op == OP_SI || (B->kind == OR_PCTL && op == OP_A));
  }
}

static int cycles_for(const or_block *B, int op, int comp) {
  if (op == OP_AC || op == OP_MONO) return B->o.nvcyc_other;
  if (comp < B->G) return B->o.nvcyc_group;
  if (comp == B->G) return B->o.nvcyc_E;
  return B->o.nvcyc_I;
}

/* out = (approximate inverse of operator (op, comp)) rhs */
static void inv_apply_internal(or_block *B, inv_t *iv, int trans, const double *rhs, double *out) {
  int n = iv->A->n;
  double *r = (double *)xmalloc((size_t)n * sizeof(double) + 8);
  double *e = (double *)xmalloc((size_t)n * sizeof(double) + 8);
  if (iv->use_jacobi) {
    for (int i = 0; i < n; ++i) out[i] = iv->jdinv[i] * rhs[i];
    for (int s = 1; s < iv->count; ++s) {
      residual(iv->A, rhs, out, r);
      for (int i = 0; i < n; ++i) out[i] = out[i] + iv->jdinv[i] * r[i];
    }
  } else if (iv->accurate && !trans) {
    /* option #3: x = 0; x += V(rhs - A x) until the relative residual <= inner_tol */
    double nr0 = 0.0;
    for (int i = 0; i < n; ++i) nr0 += rhs[i] * rhs[i];
    nr0 = sqrt(nr0);
    for (int i = 0; i < n; ++i) out[i] = 0.0;
    for (int it = 0; it < B->o.inner_maxit; ++it) {
      residual(iv->A, rhs, out, r);
      double nr = 0.0;
      for (int i = 0; i < n; ++i) nr += r[i] * r[i];
      nr = sqrt(nr);
      if (nr <= B->o.inner_tol * nr0) break;
      or_vcycle(iv->amg, r, e);
      iv->cycles++;
      for (int i = 0; i < n; ++i) out[i] = out[i] + e[i];
    }
  } else {
    iv->cycles += iv->count;
    if (trans)
      or_vcycle_T(iv->amg, rhs, out);
    else
      or_vcycle(iv->amg, rhs, out);
    for (int c = 1; c < iv->count; ++c) {
      if (trans) {
        or_csr *AT = or_transpose(iv->A);
        residual(AT, rhs, out, r);
        or_csr_free(AT);
        or_vcycle_T(iv->amg, r, e);
      } else {
        residual(iv->A, rhs, out, r);
        or_vcycle(iv->amg, r, e);
      }
      for (int i = 0; i < n; ++i) out[i] = out[i] + e[i];
    }
  }
  free(r);
  free(e);
  (void)B;
}

static void inv_apply(or_block *B, int op, int comp, const double *rhs, double *out, or_inv_cb cb, void *ctx) {
  B->ninv++;
  if (cb)
    cb(ctx, op, comp, B->N, rhs, out);
  else
    inv_apply_internal(B, &B->inv[op][comp], 0, rhs, out);
}

/* modified operator: A_a with diag -= (x[k] * y[k]) / z[k] */
static or_csr *diag_modified(const or_csr *A, const double *x, const double *y, const double *z) {
  or_csr *M = csr_copy(A);
  if (!x || !y) return M;
  for (int k = 0; k < M->n; ++k) {
    int p = diag_pos(M, k);
    double t = x[k] * y[k];
    t = t / z[k];
    M->v[p] = M->v[p] - t;
  }
  return M;
}

static double *diag_of(const or_csr *A) {
  double *d = (double *)xmalloc((size_t)A->n * sizeof(double) + 8);
  for (int i = 0; i < A->n; ++i) {
    int p = diag_pos(A, i);
    d[i] = p >= 0 ? A->v[p] : 0.0;
  }
  return d;
}

/* option #3: p = A^{-1} rhs by V-cycles until ||rhs - A p|| <= tol ||rhs|| */
static void inner_solve(const or_block *B, const or_csr *A, const or_amg *h, const double *rhs, double *p) {
  int n = A->n;
  double *r = (double *)xmalloc((size_t)n * sizeof(double) + 8);
  double *e = (double *)xmalloc((size_t)n * sizeof(double) + 8);
  double nr0 = 0.0;
  for (int i = 0; i < n; ++i) nr0 += rhs[i] * rhs[i];
  nr0 = sqrt(nr0);
  for (int i = 0; i < n; ++i) p[i] = 0.0;
  for (int it = 0; it < B->o.inner_maxit; ++it) {
    residual(A, rhs, p, r);
    double nr = 0.0;
    for (int i = 0; i < n; ++i) nr += r[i] * r[i];
    nr = sqrt(nr);
    if (nr <= B->o.inner_tol * nr0) break;
    or_vcycle(h, r, e);
    for (int i = 0; i < n; ++i) p[i] = p[i] + e[i];
  }
  free(r);
  free(e);
}

or_block *or_block_setup(const or_csr *A, int G, int N, int kind, const or_opts *o) {
  or_block *B = (or_block *)xcalloc(1, sizeof(or_block));
  int nc = G + 2, E = G, I = G + 1;
  B->G = G;
  B->N = N;
  B->nc = nc;
  B->kind = kind;
  B->o = *o;
  B->Amono = csr_copy(A);
  for (int op = 0; op < NOPS; ++op) B->inv[op] = (inv_t *)xcalloc((size_t)nc, sizeof(inv_t));
  B->t1 = (double *)xcalloc((size_t)A->n + 1, sizeof(double));
  B->t2 = (double *)xcalloc((size_t)A->n + 1, sizeof(double));
  B->t3 = (double *)xcalloc((size_t)A->n + 1, sizeof(double));
  B->t4 = (double *)xcalloc((size_t)A->n + 1, sizeof(double));
  B->t5 = (double *)xcalloc((size_t)N + 1, sizeof(double));
  B->t6 = (double *)xcalloc((size_t)N + 1, sizeof(double));
  B->dropped = (int *)xcalloc((size_t)nc * nc, sizeof(int));
  if (kind == OR_AMG) {
    inv_t *iv = &B->inv[OP_MONO][0];
    iv->A = csr_copy(A);
    iv->count = o->nvcyc_other;
    iv->amg = or_amg_setup(A, o);
    return B;
  }
  /* block extraction: rows a*N..a*N+N-1; same-block columns form A_a,
     other-block columns must sit in the same cell and form D_ab */
  B->Ab = (or_csr **)xcalloc((size_t)nc, sizeof(or_csr *));
  B->d = (double **)xcalloc((size_t)nc * nc, sizeof(double *));
  B->diag = (double **)xcalloc((size_t)nc, sizeof(double *));
  for (int a = 0; a < nc; ++a) {
    int cnt = 0;
    for (int k = 0; k < N; ++k) {
      int i = a * N + k;
      for (int p = A->rp[i]; p < A->rp[i + 1]; ++p)
        if (A->ci[p] / N == a) ++cnt;
    }
    or_csr *Aa = csr_alloc(N, N, cnt);
    int q = 0;
    for (int k = 0; k < N; ++k) {
      int i = a * N + k;
      for (int p = A->rp[i]; p < A->rp[i + 1]; ++p) {
        int bblk = A->ci[p] / N;
        if (bblk == a) {
          Aa->ci[q] = A->ci[p] - a * N;
          Aa->v[q] = A->v[p];
          ++q;
        } else {
          if (!B->d[a * nc + bblk]) B->d[a * nc + bblk] = (double *)xcalloc((size_t)N, sizeof(double));
          B->d[a * nc + bblk][k] = A->v[p];
        }
      }
      Aa->rp[k + 1] = q;
    }
    B->Ab[a] = Aa;
    B->diag[a] = diag_of(Aa);
  }
  /* Section 3.6: drop D_ab when gamma_wc^{ab} > sigma_wc */
  if (o->adaptive)
    for (int a = 0; a < nc; ++a)
      for (int b = 0; b < nc; ++b)
        if (B->d[a * nc + b] && or_gamma_wc(N, B->d[a * nc + b], B->diag[a], o->theta_wc) > o->sigma_wc) {
          free(B->d[a * nc + b]);
          B->d[a * nc + b] = NULL;
          B->dropped[a * nc + b] = 1;
        }
  double **d = B->d;
#define DV(a, b) (d[(a) * nc + (b)])
  switch (kind) {
    case OR_BD:
    case OR_BLT:
      for (int a = 0; a < nc; ++a) inv_build(B, OP_A, a, csr_copy(B->Ab[a]), cycles_for(B, OP_A, a));
      break;
    case OR_SCHUR1: {
      /* C_E-hat = A_E - D_EI diag(A_I)^{-1} D_IE;  C_g-hat = A_g - D_gE diag(C_E-hat)^{-1} D_Eg */
      inv_build(B, OP_A, I, csr_copy(B->Ab[I]), cycles_for(B, OP_A, I));
      or_csr *CE = diag_modified(B->Ab[E], DV(E, I), DV(I, E), B->diag[I]);
      double *dCE = diag_of(CE);
      if (o->opt4_steps > 0) {
        /* option #4: C_E^{-1} by the recurrence on A_E and A_I; C_E-hat only gives C_g-hat its diagonal */
        or_csr_free(CE);
        inv_build(B, OP_A, E, csr_copy(B->Ab[E]), cycles_for(B, OP_A, E));
      } else {
        inv_build(B, OP_CE, E, CE, cycles_for(B, OP_CE, E));
      }
      for (int g = 0; g < G; ++g)
        inv_build(B, OP_CG, g, diag_modified(B->Ab[g], DV(g, E), DV(E, g), dCE), cycles_for(B, OP_CG, g));
      free(dCE);
      break;
    }
    case OR_SCHUR2: {
      /* S_g-hat = A_g - D_gE diag(A_E)^{-1} D_Eg;  S_I-hat = A_I - D_IE diag(A_E)^{-1} D_EI */
      inv_build(B, OP_A, E, csr_copy(B->Ab[E]), cycles_for(B, OP_A, E));
      for (int g = 0; g < G; ++g)
        inv_build(B, OP_SG, g, diag_modified(B->Ab[g], DV(g, E), DV(E, g), B->diag[E]), cycles_for(B, OP_SG, g));
      if (o->opt4_steps > 0) /* option #4: S_I^{-1} by the recurrence on A_I and A_E */
        inv_build(B, OP_A, I, csr_copy(B->Ab[I]), cycles_for(B, OP_A, I));
      else
        inv_build(B, OP_SI, I, diag_modified(B->Ab[I], DV(I, E), DV(E, I), B->diag[E]), cycles_for(B, OP_SI, I));
      break;
    }
    case OR_PCTL: {
      for (int a = 0; a < nc; ++a) inv_build(B, OP_A, a, csr_copy(B->Ab[a]), cycles_for(B, OP_A, a));
      /* p_a = -A_a^{-1} D_aE 1 by option #3 (a = groups and I) */
      B->p = (double **)xcalloc((size_t)nc, sizeof(double *));
      double *rhs = (double *)xmalloc((size_t)N * sizeof(double) + 8);
      for (int a = 0; a < nc; ++a) {
        if (a == E) continue;
        B->p[a] = (double *)xcalloc((size_t)N, sizeof(double));
        if (!DV(a, E)) continue;
        for (int k = 0; k < N; ++k) rhs[k] = -DV(a, E)[k];
        or_amg *h = B->inv[OP_A][a].amg;
        or_amg *own = NULL;
        if (!h) h = own = or_amg_setup(B->Ab[a], o);
        inner_solve(B, B->Ab[a], h, rhs, B->p[a]);
        or_amg_free(own);
      }
      free(rhs);
      /* Eq. 3.3: A_c = sum_g P_g^T A_g P_g + A_E + P_I^T A_I P_I
                        + sum_g D_Eg P_g + sum_g P_g^T D_gE + D_EI P_I + P_I^T D_IE
         on the union of the patterns of A_g, A_E, A_I */
      int *marker = (int *)xmalloc((size_t)N * sizeof(int));
      for (int k = 0; k < N; ++k) marker[k] = -1;
      int *rp = (int *)xcalloc((size_t)N + 1, sizeof(int));
      for (int i = 0; i < N; ++i) {
        int c = 0;
        for (int a = 0; a < nc; ++a)
          for (int p = B->Ab[a]->rp[i]; p < B->Ab[a]->rp[i + 1]; ++p)
            if (marker[B->Ab[a]->ci[p]] != i) {
              marker[B->Ab[a]->ci[p]] = i;
              ++c;
            }
        rp[i + 1] = c;
      }
      for (int i = 0; i < N; ++i) rp[i + 1] += rp[i];
      or_csr *Ac = csr_alloc(N, N, rp[N]);
      memcpy(Ac->rp, rp, ((size_t)N + 1) * sizeof(int));
      free(rp);
      for (int k = 0; k < N; ++k) marker[k] = -1;
      for (int i = 0; i < N; ++i) {
        int base = Ac->rp[i], len = 0;
        for (int a = 0; a < nc; ++a)
          for (int p = B->Ab[a]->rp[i]; p < B->Ab[a]->rp[i + 1]; ++p)
            if (marker[B->Ab[a]->ci[p]] != i) {
              marker[B->Ab[a]->ci[p]] = i;
              Ac->ci[base + len++] = B->Ab[a]->ci[p];
            }
        double *tmp = Ac->v + base;
        for (int s = 0; s < len; ++s) tmp[s] = 0.0;
        sort_row(Ac->ci + base, tmp, len);
        for (int s = 0; s < len; ++s) {
          int j = Ac->ci[base + s];
          double acc = 0.0;
          for (int g = 0; g < G; ++g)
            for (int p = B->Ab[g]->rp[i]; p < B->Ab[g]->rp[i + 1]; ++p)
              if (B->Ab[g]->ci[p] == j) acc = acc + (B->p[g][i] * B->Ab[g]->v[p]) * B->p[g][j];
          for (int p = B->Ab[E]->rp[i]; p < B->Ab[E]->rp[i + 1]; ++p)
            if (B->Ab[E]->ci[p] == j) acc = acc + B->Ab[E]->v[p];
          for (int p = B->Ab[I]->rp[i]; p < B->Ab[I]->rp[i + 1]; ++p)
            if (B->Ab[I]->ci[p] == j) acc = acc + (B->p[I][i] * B->Ab[I]->v[p]) * B->p[I][j];
          if (j == i) {
            for (int g = 0; g < G; ++g)
              if (DV(E, g)) acc = acc + DV(E, g)[i] * B->p[g][i];
            for (int g = 0; g < G; ++g)
              if (DV(g, E)) acc = acc + B->p[g][i] * DV(g, E)[i];
            if (DV(E, I)) acc = acc + DV(E, I)[i] * B->p[I][i];
            if (DV(I, E)) acc = acc + B->p[I][i] * DV(I, E)[i];
          }
          tmp[s] = acc;
        }
      }
      free(marker);
      B->Ac = Ac;
      inv_build(B, OP_AC, E, csr_copy(Ac), cycles_for(B, OP_AC, E));
      break;
    }
    default:
      break;
  }
#undef DV
  return B;
}

/* t = a - d (.) v  (d may be NULL: t = a) */
static void hsub(int N, const double *a, const double *d, const double *v, double *t) {
  for (int k = 0; k < N; ++k) t[k] = d ? a[k] - d[k] * v[k] : a[k];
}
/* t += d (.) v */
static void hacc(int N, const double *d, const double *v, double *t) {
  if (!d) return;
  for (int k = 0; k < N; ++k) t[k] = t[k] + d[k] * v[k];
}

/* option #4 (Section 3.5): w = S^{-1} q for S = A_a - D_ab A_b^{-1} D_ba, approximated by
   K = opt4_steps steps of w^(0) = 0, w^(k+1) = A_a^{-1}(q + D_ab A_b^{-1} D_ba w^(k)).
   The first step is w^(1) = A_a^{-1} q (its inner term is zero). */
static void opt4_apply(or_block *B, int a, int b, const double *q, double *w, or_inv_cb cb, void *ctx) {
  int N = B->N, nc = B->nc;
  const double *dab = B->d[a * nc + b], *dba = B->d[b * nc + a];
  double *s = B->t5, *u = B->t6;
  inv_apply(B, OP_A, a, q, w, cb, ctx);
  for (int k = 1; k < B->o.opt4_steps; ++k) {
    for (int i = 0; i < N; ++i) s[i] = dba ? dba[i] * w[i] : 0.0;
    inv_apply(B, OP_A, b, s, u, cb, ctx);
    for (int i = 0; i < N; ++i) s[i] = dab ? q[i] + dab[i] * u[i] : q[i];
    inv_apply(B, OP_A, a, s, w, cb, ctx);
  }
}

void or_block_apply(or_block *B, const double *v, double *z, or_inv_cb cb, void *ctx) {
  int G = B->G, N = B->N, nc = B->nc, E = G, I = G + 1;
  double **d = B->d;
  double *t = B->t1, *u = B->t2, *wEs = B->t3, *wIs = B->t4;
#define DV(a, b) (d[(a) * nc + (b)])
#define BLK(x, a) ((x) + (size_t)(a) * N)
  B->ninv = 0;
  B->nmatvec = 0;
  switch (B->kind) {
    case OR_AMG:
      inv_apply(B, OP_MONO, 0, v, z, cb, ctx);
      break;
    case OR_BD:
      for (int a = 0; a < nc; ++a) inv_apply(B, OP_A, a, BLK(v, a), BLK(z, a), cb, ctx);
      break;
    case OR_BLT:
      /* lower triangular: groups, then E, then I */
      for (int g = 0; g < G; ++g) inv_apply(B, OP_A, g, BLK(v, g), BLK(z, g), cb, ctx);
      memcpy(t, BLK(v, E), (size_t)N * sizeof(double));
      for (int g = 0; g < G; ++g)
        if (DV(E, g))
          for (int k = 0; k < N; ++k) t[k] = t[k] - DV(E, g)[k] * BLK(z, g)[k];
      inv_apply(B, OP_A, E, t, BLK(z, E), cb, ctx);
      hsub(N, BLK(v, I), DV(I, E), BLK(z, E), t);
      inv_apply(B, OP_A, I, t, BLK(z, I), cb, ctx);
      break;
    case OR_SCHUR1:
      /* 1: w_I* = A_I^{-1} b_I */
      inv_apply(B, OP_A, I, BLK(v, I), wIs, cb, ctx);
      /* 2: w_E* = C_E^{-1}(b_E - D_EI w_I*) */
      hsub(N, BLK(v, E), DV(E, I), wIs, t);
      if (B->o.opt4_steps > 0)
        opt4_apply(B, E, I, t, wEs, cb, ctx);
      else
        inv_apply(B, OP_CE, E, t, wEs, cb, ctx);
      /* 3: w_g = C_g^{-1}(b_g - D_gE w_E*) */
      for (int g = 0; g < G; ++g) {
        hsub(N, BLK(v, g), DV(g, E), wEs, t);
        inv_apply(B, OP_CG, g, t, BLK(z, g), cb, ctx);
      }
      /* 4: w_E = w_E* - C_E^{-1} sum_g D_Eg w_g */
      for (int k = 0; k < N; ++k) t[k] = 0.0;
      for (int g = 0; g < G; ++g) hacc(N, DV(E, g), BLK(z, g), t);
      if (B->o.opt4_steps > 0)
        opt4_apply(B, E, I, t, u, cb, ctx);
      else
        inv_apply(B, OP_CE, E, t, u, cb, ctx);
      for (int k = 0; k < N; ++k) BLK(z, E)[k] = wEs[k] - u[k];
      /* 5: w_I = w_I* - A_I^{-1} D_IE w_E */
      for (int k = 0; k < N; ++k) t[k] = 0.0;
      hacc(N, DV(I, E), BLK(z, E), t);
      inv_apply(B, OP_A, I, t, u, cb, ctx);
      for (int k = 0; k < N; ++k) BLK(z, I)[k] = wIs[k] - u[k];
      break;
    case OR_SCHUR2:
      /* 1: w_E* = A_E^{-1} b_E */
      inv_apply(B, OP_A, E, BLK(v, E), wEs, cb, ctx);
      /* 2: w_g = S_g^{-1}(b_g - D_gE w_E*), w_I = S_I^{-1}(b_I - D_IE w_E*) */
      for (int g = 0; g < G; ++g) {
        hsub(N, BLK(v, g), DV(g, E), wEs, t);
        inv_apply(B, OP_SG, g, t, BLK(z, g), cb, ctx);
      }
      hsub(N, BLK(v, I), DV(I, E), wEs, t);
      if (B->o.opt4_steps > 0)
        opt4_apply(B, I, E, t, BLK(z, I), cb, ctx);
      else
        inv_apply(B, OP_SI, I, t, BLK(z, I), cb, ctx);
      /* 3: w_E = w_E* - A_E^{-1}(sum_g D_Eg w_g + D_EI w_I) */
      for (int k = 0; k < N; ++k) t[k] = 0.0;
      for (int g = 0; g < G; ++g) hacc(N, DV(E, g), BLK(z, g), t);
      hacc(N, DV(E, I), BLK(z, I), t);
      inv_apply(B, OP_A, E, t, u, cb, ctx);
      for (int k = 0; k < N; ++k) BLK(z, E)[k] = wEs[k] - u[k];
      break;
    case OR_PCTL: {
      /* 1: block relaxation, E first (coarse points), then the others */
      inv_apply(B, OP_A, E, BLK(v, E), BLK(z, E), cb, ctx);
      for (int a = 0; a < nc; ++a) {
        if (a == E) continue;
        hsub(N, BLK(v, a), DV(a, E), BLK(z, E), t);
        inv_apply(B, OP_A, a, t, BLK(z, a), cb, ctx);
      }
      /* 2: r = b - A w block row by block row, r_c = P^T r, A_c w_c = r_c */
      double *rc = wEs, *wc = wIs;
      for (int k = 0; k < N; ++k) rc[k] = 0.0;
      for (int a = 0; a < nc; ++a) {
        residual(B->Ab[a], BLK(v, a), BLK(z, a), t);
        B->nmatvec++;
        for (int b = 0; b < nc; ++b)
          if (b != a && DV(a, b))
            for (int k = 0; k < N; ++k) t[k] = t[k] - DV(a, b)[k] * BLK(z, b)[k];
        if (a == E)
          for (int k = 0; k < N; ++k) rc[k] = rc[k] + t[k];
        else
          for (int k = 0; k < N; ++k) rc[k] = rc[k] + B->p[a][k] * t[k];
      }
      inv_apply(B, OP_AC, E, rc, wc, cb, ctx);
      /* 3: w += P w_c */
      for (int a = 0; a < nc; ++a) {
        if (a == E)
          for (int k = 0; k < N; ++k) BLK(z, a)[k] = BLK(z, a)[k] + wc[k];
        else
          for (int k = 0; k < N; ++k) BLK(z, a)[k] = BLK(z, a)[k] + B->p[a][k] * wc[k];
      }
      break;
    }
    default:
      break;
  }
#undef DV
#undef BLK
}

/* transposed apply: supported for the monolithic AMG and block-diagonal kinds */
void or_block_apply_T(or_block *B, const double *v, double *z) {
  int N = B->N, nc = B->nc;
  B->ninv = 0;
  if (B->kind == OR_AMG) {
    B->ninv = 1;
    inv_apply_internal(B, &B->inv[OP_MONO][0], 1, v, z);
  } else if (B->kind == OR_BD) {
    for (int a = 0; a < nc; ++a) {
      B->ninv++;
      inv_apply_internal(B, &B->inv[OP_A][a], 1, v + (size_t)a * N, z + (size_t)a * N);
    }
  } else {
    fprintf(stderr, "oracle: transposed apply only for AMG and BD\n");
    abort();
  }
}

int or_block_ninv(const or_block *B) { return B->ninv; }
int or_block_nmatvec(const or_block *B) { return B->nmatvec; }
int or_block_dropped(const or_block *B, int a, int b) { return B->dropped ? B->dropped[a * B->nc + b] : 0; }
int or_block_use_jacobi(const or_block *B, int op, int comp) { return B->inv[op][comp].use_jacobi; }
const or_amg *or_block_amg(const or_block *B, int op, int comp) { return B->inv[op][comp].amg; }
long or_block_cycles(const or_block *B, int op, int comp) { return B->inv[op][comp].cycles; }

const double *or_block_vec(const or_block *B, int which, int comp) {
  if (which == 0) return B->p ? B->p[comp] : NULL;
  return B->diag ? B->diag[comp] : NULL;
}
const or_csr *or_block_Ac(const or_block *B) { return B->Ac; }

void or_block_free(or_block *B) {
  if (!B) return;
  for (int op = 0; op < NOPS; ++op) {
    for (int c = 0; c < B->nc; ++c) {
      or_csr_free(B->inv[op][c].A);
      or_amg_free(B->inv[op][c].amg);
      free(B->inv[op][c].jdinv);
    }
    free(B->inv[op]);
  }
  if (B->Ab)
    for (int a = 0; a < B->nc; ++a) {
      or_csr_free(B->Ab[a]);
      free(B->diag[a]);
    }
  if (B->d)
    for (int a = 0; a < B->nc * B->nc; ++a) free(B->d[a]);
  if (B->p)
    for (int a = 0; a < B->nc; ++a) free(B->p[a]);
  free(B->Ab);
  free(B->diag);
  free(B->d);
  free(B->p);
  free(B->dropped);
  or_csr_free(B->Ac);
  or_csr_free(B->Amono);
  free(B->t1);
  free(B->t2);
  free(B->t3);
  free(B->t4);
  free(B->t5);
  free(B->t6);
  free(B);
}

/* ------------------------------------------------------------------ */
/* Right-preconditioned flexible GMRES(m) (Saad 1993) with modified     */
/* Gram-Schmidt and Givens rotations.  Converged when the relative      */
/* residual ||b - A x|| / ||b|| <= tol (Section 4 stopping rule); the   */
/* Arnoldi estimate ends a cycle, the true residual decides.            */
/* Iterations count preconditioner applications.                        */
/* Returns 0 converged, 1 iteration cap reached, 3 non-finite residual. */
/* ------------------------------------------------------------------ */
static double dot(int n, const double *a, const double *b) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

int or_fgmres(const or_csr *A0, or_block *M, int transpose, const double *b, double *x, double tol, int m,
              int maxit, int *iters, double *relres, double *hist) {
  int n = A0->n;
  or_csr *AT = transpose ? or_transpose(A0) : NULL;
  const or_csr *A = transpose ? AT : A0;
  double bnorm = sqrt(dot(n, b, b));
  *iters = 0;
  if (bnorm == 0.0) {
    for (int i = 0; i < n; ++i) x[i] = 0.0;
    *relres = 0.0;
    or_csr_free(AT);
    return 0;
  }
  double *V = (double *)xmalloc((size_t)(m + 1) * n * sizeof(double));
  double *Z = (double *)xmalloc((size_t)m * n * sizeof(double));
  double *H = (double *)xcalloc((size_t)(m + 1) * m, sizeof(double));
  double *cs = (double *)xcalloc((size_t)m, sizeof(double));
  double *sn = (double *)xcalloc((size_t)m, sizeof(double));
  double *g = (double *)xcalloc((size_t)m + 1, sizeof(double));
  double *y = (double *)xcalloc((size_t)m, sizeof(double));
  double *r = (double *)xmalloc((size_t)n * sizeof(double));
  double *w = (double *)xmalloc((size_t)n * sizeof(double));
  int it = 0, status = 1, broke = 0;
#define Hm(i, j) H[(size_t)(i) * m + (j)]
  for (;;) {
    residual(A, b, x, r);
    double beta = sqrt(dot(n, r, r));
    *relres = beta / bnorm;
    if (!isfinite(beta)) {
      status = 3;
      break;
    }
    if (beta <= tol * bnorm) {
      status = 0;
      break;
    }
    /* an Arnoldi breakdown (h_{j+1,j} = 0) with a nonsingular Hessenberg
       matrix gives the exact solution of the preconditioned system; when the
       true residual still misses the tolerance, restarting from the same
       data cannot do better: report the breakdown */
    if (broke) {
      status = 2;
      break;
    }
    if (it >= maxit) {
      status = 1;
      break;
    }
    for (int i = 0; i < n; ++i) V[i] = r[i] / beta;
    for (int i = 0; i <= m; ++i) g[i] = 0.0;
    g[0] = beta;
    int j = 0;
    while (j < m) {
      double *vj = V + (size_t)j * n, *zj = Z + (size_t)j * n;
      if (transpose)
        or_block_apply_T(M, vj, zj);
      else if (M)
        or_block_apply(M, vj, zj, NULL, NULL);
      else
        memcpy(zj, vj, (size_t)n * sizeof(double));
      ++it;
      or_spmv(A, zj, w);
      for (int i = 0; i <= j; ++i) {
        double h = dot(n, w, V + (size_t)i * n);
        Hm(i, j) = h;
        const double *vi = V + (size_t)i * n;
        for (int k = 0; k < n; ++k) w[k] = w[k] - h * vi[k];
      }
      double hn = sqrt(dot(n, w, w));
      Hm(j + 1, j) = hn;
      if (hn != 0.0)
        for (int k = 0; k < n; ++k) V[(size_t)(j + 1) * n + k] = w[k] / hn;
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
        double tt = sqrt(h1 * h1 + h2 * h2);
        cs[j] = h1 / tt;
        sn[j] = h2 / tt;
      }
      Hm(j, j) = cs[j] * h1 + sn[j] * h2;
      Hm(j + 1, j) = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      if (hist) hist[it - 1] = fabs(g[j + 1]) / bnorm;
      ++j;
      if (hn == 0.0) broke = 1;
      if (fabs(g[j]) <= tol * bnorm || hn == 0.0 || it >= maxit || !isfinite(g[j])) break;
    }
    /* a zero on the diagonal of the rotated Hessenberg matrix: the least-squares
       problem is singular (breakdown without a solution); x keeps its value */
    int singular = 0;
    for (int i = 0; i < j; ++i)
      if (Hm(i, i) == 0.0) singular = 1;
    if (singular) {
      status = 2;
      break;
    }
    /* y = H(0:j,0:j)^{-1} g(0:j); x += Z y */
    for (int i = j - 1; i >= 0; --i) {
      double s = g[i];
      for (int k = i + 1; k < j; ++k) s -= Hm(i, k) * y[k];
      y[i] = s / Hm(i, i);
    }
    for (int i = 0; i < j; ++i) {
      const double *zi = Z + (size_t)i * n;
      for (int k = 0; k < n; ++k) x[k] = x[k] + y[i] * zi[k];
    }
  }
#undef Hm
  *iters = it;
  free(V);
  free(Z);
  free(H);
  free(cs);
  free(sn);
  free(g);
  free(y);
  free(r);
  free(w);
  or_csr_free(AT);
  return status;
}

void or_grad_vals(const or_csr *A, const double *x, const double *lambda, double *g) {
  for (int i = 0; i < A->n; ++i)
    for (int p = A->rp[i]; p < A->rp[i + 1]; ++p) g[p] = -lambda[i] * x[A->ci[p]];
}
