/*
 * amg_oracle.c -- plain, slow, single-threaded FP64 reference of
 * classical-AMG-preconditioned conjugate gradients (Chronos, arXiv 2102.07417).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle against which the CUDA
 * library is checked.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header,
 * table or helper with the CUDA library and never calls it.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (no FMA
 * contraction, so every product is rounded before it is added; the
 * canonical evaluation orders stated below are then exact specifications).
 *
 * What it follows, step by step:
 *   - strength of connection: Sec. 2.2, classical measure (Eq. cla) with the
 *     threshold filter; the printed denominator is garbled, and the reading
 *     taken is the Ruge-Stueben one: j strongly influences i iff
 *     -a_ij >= theta * max_{k != i}(-a_ik), the maximum taken over row i.
 *   - C/F splitting: PMIS (Sec. 2.2, cited De Sterck-Yang-Heys), seeded by a
 *     counter-based SplitMix64 stream; rounds are synchronous.
 *   - prolongation P = [W; I] (Eq. prolOperator) with W from direct
 *     interpolation (Stueben's direct formula; the paper names no
 *     distance-one direct formula, so this is the reading taken).
 *   - R = P^T and A_c = P^T A P (Eq. AcDef), computed as R (A P) in a
 *     canonical order (below).
 *   - Algorithm 1 (AMG_SetUp) with a dense Cholesky on the last level.
 *   - Algorithm 2 (AMG_Apply, V-cycle) with the smoother
 *     S = I - omega M^{-1} A (Eq. smoother): damped Jacobi (M = D), or the
 *     factored sparse approximate inverse M^{-1} = G^T G with G lower
 *     triangular (Eq. smo), G on the static pattern of lower(A).
 *   - PCG from x0 with the stopping rule ||r_k|| < rtol ||b|| on the
 *     recursively updated residual (Sec. 4); standard or flexible
 *     (Polak-Ribiere) beta.
 *
 * Canonical orders (needed for bit-exact hierarchies, since a one-ulp change
 * at an exact strength tie changes the next coarse grid):
 *   (A P)_{iJ}   = sum over j ascending in row i of A of  a_ij * P_jJ
 *   (A_c)_{IJ}   = sum over i ascending in row I of R of  R_Ii * (AP)_iJ
 *   each product rounded, then added left to right starting from 0.
 *   Interpolation sums run over the row in ascending column order.
 *
 * Parity pins for every function are in tests/test_oracle_pins.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_NOT_SPD (-2)
#define OR_ERR_BREAKDOWN (-3)
#define OR_ERR_NO_CONVERGENCE (-4)
#define OR_ERR_SETUP (-5)
#define OR_ERR_MEM (-6)

#define OR_MAX_LEVELS 40
#define OR_MAX_DENSE 4096

typedef struct {
  int n;
  int nnz;
  int *rp;
  int *ci;
  double *v;
} or_csr;

typedef struct {
  int nlevels;
  or_csr A[OR_MAX_LEVELS];
  or_csr P[OR_MAX_LEVELS]; /* P[k]: n_k x n_{k+1}, k < nlevels-1 */
  or_csr R[OR_MAX_LEVELS]; /* R[k] = P[k]^T */
  signed char *cf[OR_MAX_LEVELS];
  unsigned char *S[OR_MAX_LEVELS];
  or_csr G[OR_MAX_LEVELS];     /* FSAI factor of level k (smoother 1), k < nlevels-1 */
  double *L;                   /* dense Cholesky factor of the last level, row-major */
  int nL;
  double omega;
  int nu1, nu2;
  int smoother;                /* 0 damped Jacobi, 1 FSAI */
  /* work vectors per level */
  double *wr[OR_MAX_LEVELS], *wy[OR_MAX_LEVELS], *wz[OR_MAX_LEVELS], *ws[OR_MAX_LEVELS];
} or_hier;

static void csr_free(or_csr *m) {
  free(m->rp);
  free(m->ci);
  free(m->v);
  memset(m, 0, sizeof(*m));
}

static int csr_alloc(or_csr *m, int n, int nnz) {
  m->n = n;
  m->nnz = nnz;
  m->rp = (int *)calloc((size_t)n + 1, sizeof(int));
  m->ci = (int *)malloc(((size_t)nnz + 1) * sizeof(int));
  m->v = (double *)malloc(((size_t)nnz + 1) * sizeof(double));
  return (m->rp && m->ci && m->v) ? OR_OK : OR_ERR_MEM;
}

/* ------------------------------------------------------------------ */
/* Input validation: rows ascending, columns in range and strictly       */
/* ascending, a positive diagonal present in every row.                  */
/* ------------------------------------------------------------------ */
int or_check_csr(int n, const int *rp, const int *ci, const double *a) {
  if (n < 1 || rp[0] != 0) return OR_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    if (rp[i + 1] < rp[i]) return OR_ERR_ARG;
    int has_diag = 0;
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      if (ci[p] < 0 || ci[p] >= n) return OR_ERR_ARG;
      if (p > rp[i] && ci[p] <= ci[p - 1]) return OR_ERR_ARG;
      if (!isfinite(a[p])) return OR_ERR_ARG; /* values must be finite */
      if (ci[p] == i) {
        has_diag = 1;
        if (!(a[p] > 0.0)) return OR_ERR_NOT_SPD;
      }
    }
    if (!has_diag) return OR_ERR_ARG;
  }
  return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Strength of connection (Sec. 2.2, Eq. cla read as Ruge-Stueben, with   */
/* the threshold filter).  S[p] = 1 iff column ci[p] strongly influences  */
/* row i:  ci[p] != i  and  -a[p] >= theta * m_i,  m_i = max_{k!=i} -a_ik, */
/* and only when m_i > 0.                                                 */
/* ------------------------------------------------------------------ */
int or_strength(int n, const int *rp, const int *ci, const double *a, double theta, unsigned char *S) {
  for (int i = 0; i < n; ++i) {
    double m = 0.0;
    int have = 0;
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      if (ci[p] == i) continue;
      double t = -a[p];
      if (!have || t > m) m = t;
      have = 1;
    }
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      S[p] = 0;
      if (!have || !(m > 0.0) || ci[p] == i) continue;
      if (-a[p] >= theta * m) S[p] = 1;
    }
  }
  return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Nodal (block) strength for systems with bs unknowns per node, numbered */
/* node-major (unknown i belongs to node i / bs, component i % bs).  This */
/* is the block form of the scaled measure (Eq. sco, Sec. 2.2) with       */
/* Frobenius norms of the bs x bs blocks A_IJ:                            */
/*   s_IJ = ||A_IJ||_F / sqrt(||A_II||_F ||A_JJ||_F),                     */
/*   J strongly influences I iff J != I, m_I = max_{K != I} s_IK > 0 and   */
/*   s_IJ >= theta * m_I.                                                 */
/* ||A_IJ||_F^2 sums a^2 over the rows of node I in order and, within a   */
/* row, over the columns of node J in ascending order.                    */
/* Outputs: the node graph (Nrp[nn + 1], Nci[<= nnz], node J present iff  */
/* some row of I has a column of J), its strength SN, and the unknown-    */
/* wise strength S[p] = 1 iff column ci[p] has the row's component, lies  */
/* in another node J, and SN(I, J).                                       */
/* ------------------------------------------------------------------ */
static int cmp_int(const void *x, const void *y);

static int node_pos(const int *Nrp, const int *Nci, int I, int J) {
  int lo = Nrp[I], hi = Nrp[I + 1] - 1;
  while (lo <= hi) {
    int mid = (lo + hi) / 2;
    if (Nci[mid] == J) return mid;
    if (Nci[mid] < J) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

int or_block_strength(int n, const int *rp, const int *ci, const double *a, int bs, double theta, int *nn_out,
                      int *Nrp, int *Nci, unsigned char *SN, unsigned char *S) {
  if (bs < 1 || n % bs) return OR_ERR_ARG;
  int nn = n / bs;
  *nn_out = nn;
  int *tmp = (int *)malloc(((size_t)rp[n] + 1) * sizeof(int));
  if (!tmp) return OR_ERR_MEM;
  Nrp[0] = 0;
  for (int I = 0; I < nn; ++I) {
    int cnt = 0;
    for (int c = 0; c < bs; ++c)
      for (int p = rp[I * bs + c]; p < rp[I * bs + c + 1]; ++p) tmp[cnt++] = ci[p] / bs;
    qsort(tmp, (size_t)cnt, sizeof(int), cmp_int);
    int u = 0;
    for (int t = 0; t < cnt; ++t)
      if (u == 0 || tmp[t] != tmp[u - 1]) tmp[u++] = tmp[t];
    memcpy(Nci + Nrp[I], tmp, (size_t)u * sizeof(int));
    Nrp[I + 1] = Nrp[I] + u;
  }
  free(tmp);
  int nne = Nrp[nn];
  double *F = (double *)malloc(((size_t)nne + 1) * sizeof(double));
  double *dn = (double *)calloc((size_t)nn + 1, sizeof(double));
  if (!F || !dn) {
    free(F); free(dn);
    return OR_ERR_MEM;
  }
  for (int I = 0; I < nn; ++I) {
    for (int e = Nrp[I]; e < Nrp[I + 1]; ++e) {
      int J = Nci[e];
      double f2 = 0.0;
      for (int c = 0; c < bs; ++c)
        for (int p = rp[I * bs + c]; p < rp[I * bs + c + 1]; ++p)
          if (ci[p] / bs == J) f2 += a[p] * a[p];
      F[e] = sqrt(f2);
      if (J == I) dn[I] = F[e];
    }
  }
  for (int I = 0; I < nn; ++I) {
    double m = 0.0;
    for (int e = Nrp[I]; e < Nrp[I + 1]; ++e) {
      int J = Nci[e];
      double den = sqrt(dn[I] * dn[J]);
      F[e] = (den > 0.0) ? F[e] / den : 0.0; /* F now holds s_IJ */
      if (J != I && F[e] > m) m = F[e];
    }
    for (int e = Nrp[I]; e < Nrp[I + 1]; ++e)
      SN[e] = (Nci[e] != I && m > 0.0 && F[e] >= theta * m) ? 1 : 0;
  }
  for (int i = 0; i < n; ++i) {
    int I = i / bs;
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      int j = ci[p], J = j / bs;
      S[p] = (j % bs == i % bs && J != I && SN[node_pos(Nrp, Nci, I, J)]) ? 1 : 0;
    }
  }
  free(F); free(dn);
  return OR_OK;
}

/* ------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea & Flood 2014), used counter-based:             */
/* output number c (c = 1, 2, ...) of the generator seeded with `seed` is  */
/* mix(seed + c * 0x9E3779B97F4A7C15).  The PMIS measure of point i on     */
/* level k takes c = (k << 32) + i + 1 and maps the top 53 bits to [0,1).  */
/* ------------------------------------------------------------------ */
uint64_t or_splitmix64(uint64_t seed, uint64_t c) {
  uint64_t z = seed + c * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

double or_pmis_random(uint64_t seed, int level, int i) {
  uint64_t c = ((uint64_t)(uint32_t)level << 32) + (uint64_t)(uint32_t)i + 1ULL;
  return (double)(or_splitmix64(seed, c) >> 11) * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------------------------------ */
/* PMIS C/F splitting (Sec. 2.2; De Sterck, Yang & Heys).                 */
/*   lambda_i = |S_i^T| + u_i ,  S_i^T = { j : i in S_j }.                 */
/*   Points with lambda_i < 1 (influencing nobody) start as F.            */
/*   Each round, with the state frozen at the round's start:               */
/*     an undecided i becomes C if it beats every undecided j in           */
/*     S_i u S_i^T (beats: larger lambda, ties broken by larger index);    */
/*     then every undecided i with S_i meeting the new C points becomes F. */
/* or_pmis_rounds takes the measures as input and stops after max_rounds  */
/* rounds (max_rounds < 0: until no point is undecided); state[i] = 1 C,  */
/* 0 F, -1 still undecided; *rounds_out (may be NULL) = rounds run.       */
/* or_pmis draws the measures from the counter-based stream and writes    */
/* cf[i] = 1 for C, 0 for F.                                              */
/* ------------------------------------------------------------------ */
enum { ST_U = 0, ST_C = 1, ST_F = 2, ST_NEWC = 3 };

/* the state a competitor j had at the start of the round: undecided */
static int competes(const unsigned char *st, int j) { return st[j] == ST_U || st[j] == ST_NEWC; }

/* i beats j: larger measure, equal measures broken by the larger index */
static int beats(const double *lam, int i, int j) { return lam[i] > lam[j] || (lam[i] == lam[j] && i > j); }

int or_pmis_rounds(int n, const int *rp, const int *ci, const unsigned char *S, const double *lam, int max_rounds,
                   signed char *state, int *rounds_out) {
  int *tcnt = (int *)calloc((size_t)n + 1, sizeof(int));
  unsigned char *st = (unsigned char *)malloc((size_t)n + 1);
  if (!tcnt || !st) {
    free(tcnt); free(st);
    return OR_ERR_MEM;
  }
  /* S^T as CSR: for each strong entry (j -> c) of row j, row c of S^T gets j */
  for (int j = 0; j < n; ++j)
    for (int p = rp[j]; p < rp[j + 1]; ++p)
      if (S[p]) tcnt[ci[p] + 1]++;
  for (int i = 0; i < n; ++i) tcnt[i + 1] += tcnt[i];
  int ntr = tcnt[n];
  int *tcol = (int *)malloc(((size_t)ntr + 1) * sizeof(int));
  int *fill = (int *)malloc(((size_t)n + 1) * sizeof(int));
  if (!tcol || !fill) {
    free(tcnt); free(st); free(tcol); free(fill);
    return OR_ERR_MEM;
  }
  for (int i = 0; i < n; ++i) fill[i] = tcnt[i];
  for (int j = 0; j < n; ++j)
    for (int p = rp[j]; p < rp[j + 1]; ++p)
      if (S[p]) tcol[fill[ci[p]]++] = j;

  for (int i = 0; i < n; ++i) st[i] = (lam[i] < 1.0) ? ST_F : ST_U;
  int rounds = 0;
  while (max_rounds < 0 || rounds < max_rounds) {
    int undecided = 0;
    for (int i = 0; i < n; ++i) undecided += (st[i] == ST_U);
    if (!undecided) break;
    ++rounds;
    /* selection: local maxima of lambda among undecided strong neighbours */
    for (int i = 0; i < n; ++i) {
      if (st[i] != ST_U) continue;
      int is_max = 1;
      for (int p = rp[i]; p < rp[i + 1] && is_max; ++p) /* j in S_i */
        if (S[p] && competes(st, ci[p]) && !beats(lam, i, ci[p])) is_max = 0;
      for (int q = tcnt[i]; q < tcnt[i + 1] && is_max; ++q) /* j in S_i^T */
        if (competes(st, tcol[q]) && !beats(lam, i, tcol[q])) is_max = 0;
      if (is_max) st[i] = ST_NEWC;
    }
    /* undecided points that depend strongly on a new C point (S_i meets it) become F */
    for (int i = 0; i < n; ++i) {
      if (st[i] != ST_U) continue;
      for (int p = rp[i]; p < rp[i + 1]; ++p)
        if (S[p] && st[ci[p]] == ST_NEWC) {
          st[i] = ST_F;
          break;
        }
    }
    for (int i = 0; i < n; ++i)
      if (st[i] == ST_NEWC) st[i] = ST_C;
  }
  for (int i = 0; i < n; ++i) state[i] = (st[i] == ST_C) ? 1 : (st[i] == ST_F) ? 0 : -1;
  if (rounds_out) *rounds_out = rounds;
  free(tcnt); free(st); free(tcol); free(fill);
  return OR_OK;
}

int or_pmis(int n, const int *rp, const int *ci, const unsigned char *S, uint64_t seed, int level,
            signed char *cf) {
  int *deg = (int *)calloc((size_t)n + 1, sizeof(int));
  double *lam = (double *)malloc(((size_t)n + 1) * sizeof(double));
  if (!deg || !lam) {
    free(deg); free(lam);
    return OR_ERR_MEM;
  }
  for (int j = 0; j < n; ++j) /* |S_i^T|: the points that i strongly influences */
    for (int p = rp[j]; p < rp[j + 1]; ++p)
      if (S[p]) deg[ci[p]]++;
  for (int i = 0; i < n; ++i) lam[i] = (double)deg[i] + or_pmis_random(seed, level, i);
  int st = or_pmis_rounds(n, rp, ci, S, lam, -1, cf, NULL);
  free(deg); free(lam);
  return st;
}

/* ------------------------------------------------------------------ */
/* Direct interpolation, P = [W; I] in the original ordering             */
/* (Eq. prolOperator).  Coarse index of a C point = its rank among the C  */
/* points.  C row: a single unit entry.  F row i, with P_i = C n S_i and  */
/* N_i the off-diagonal neighbours (sums in ascending column order):      */
/*   alpha = sum_{N_i} a^- / sum_{P_i} a^-,  beta = sum_{N_i} a^+ / sum_{P_i} a^+ */
/*   at = a_ii + sum_{N_i} a^+  if P_i has no positive entry, else a_ii    */
/*   w_ij = -(alpha a_ij) / at  (a_ij < 0),  -(beta a_ij) / at  (a_ij > 0)  */
/* (the product rounded, negated, then divided: one division per weight)  */
/* Empty P_i gives an empty row.  Capacity `cap` bounds nnz(P).           */
/* ------------------------------------------------------------------ */
/* Systems (block size bs > 1, unknowns numbered node-major): unknown-wise  */
/* interpolation.  Row i only sees the columns of its own component        */
/* (j % bs == i % bs): N_i, the sums and the diagonal come from those.     */
static int direct_interp(int n, const int *rp, const int *ci, const double *a, const unsigned char *S,
                         const signed char *cf, int bs, int *cidx, int *nc_out, int *Prp, int *Pci, double *Pv,
                         long long cap);

int or_direct_interp(int n, const int *rp, const int *ci, const double *a, const unsigned char *S,
                     const signed char *cf, int *cidx, int *nc_out, int *Prp, int *Pci, double *Pv,
                     long long cap) {
  return direct_interp(n, rp, ci, a, S, cf, 1, cidx, nc_out, Prp, Pci, Pv, cap);
}

int or_direct_interp_bs(int n, const int *rp, const int *ci, const double *a, const unsigned char *S,
                        const signed char *cf, int bs, int *cidx, int *nc_out, int *Prp, int *Pci, double *Pv,
                        long long cap) {
  if (bs < 1 || n % bs) return OR_ERR_ARG;
  return direct_interp(n, rp, ci, a, S, cf, bs, cidx, nc_out, Prp, Pci, Pv, cap);
}

static int direct_interp(int n, const int *rp, const int *ci, const double *a, const unsigned char *S,
                         const signed char *cf, int bs, int *cidx, int *nc_out, int *Prp, int *Pci, double *Pv,
                         long long cap) {
  int nc = 0;
  for (int i = 0; i < n; ++i) cidx[i] = cf[i] ? nc++ : -1;
  *nc_out = nc;
  long long pos = 0;
  Prp[0] = 0;
  for (int i = 0; i < n; ++i) {
    if (cf[i]) {
      if (pos + 1 > cap) return OR_ERR_MEM;
      Pci[pos] = cidx[i];
      Pv[pos] = 1.0;
      ++pos;
      Prp[i + 1] = (int)pos;
      continue;
    }
    double aii = 0.0, sn_neg = 0.0, sn_pos = 0.0, sp_neg = 0.0, sp_pos = 0.0;
    int np = 0;
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      int j = ci[p];
      double v = a[p];
      if (j % bs != i % bs) continue; /* another component: not a neighbour here */
      if (j == i) {
        aii = v;
        continue;
      }
      if (v < 0.0) sn_neg += v;
      if (v > 0.0) sn_pos += v;
      if (S[p] && cf[j]) {
        ++np;
        if (v < 0.0) sp_neg += v;
        if (v > 0.0) sp_pos += v;
      }
    }
    if (np > 0) {
      double alpha = (sp_neg != 0.0) ? sn_neg / sp_neg : 0.0;
      double beta = (sp_pos != 0.0) ? sn_pos / sp_pos : 0.0;
      double at = (sp_pos != 0.0) ? aii : aii + sn_pos;
      if (pos + np > cap) return OR_ERR_MEM;
      for (int p = rp[i]; p < rp[i + 1]; ++p) {
        int j = ci[p];
        if (j == i || !S[p] || !cf[j]) continue;
        double v = a[p], w = 0.0;
        if (v < 0.0) w = -(alpha * v) / at;
        if (v > 0.0) w = -(beta * v) / at;
        Pci[pos] = cidx[j];
        Pv[pos] = w;
        ++pos;
      }
    }
    Prp[i + 1] = (int)pos;
  }
  return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Extended+i interpolation (Sec. 2.3, the distance-two formula; De Sterck, */
/* Falgout, Nolting & Yang).  Reading of the printed formula:              */
/*   C_i^S, F_i^S: strong C / F neighbours of i; the interpolatory set is   */
/*   Chat_i = C_i^S u (union over k in F_i^S of C_k^S);                     */
/*   abar_kl = a_kl when its sign differs from a_kk's (a_kk > 0: a_kl < 0),  */
/*   else 0;  d_k = sum over l in row k with l in Chat_i u {i} of abar_kl;   */
/*   at = a_ii + sum over weak n not in Chat_i of a_in                      */
/*             + sum over k in F_i^S of (a_ik abar_ki) / d_k ;              */
/*   w_ij = -(a_ij + sum over k in F_i^S of (a_ik abar_kj) / d_k) / at,     */
/*   j in Chat_i (a_ij = 0 when j is not a neighbour).                      */
/* Canonical evaluation (the GPU follows it bit for bit): d_k over row k in  */
/* ascending l; at from a_ii over row i's off-diagonals in ascending order   */
/* (an F_i^S term (a_ik abar_ki) / d_k or a weak a_in as the entry calls    */
/* for); each numerator from a_ij, adding the k terms in ascending k; terms  */
/* with abar_kj = 0 are skipped; a strong F neighbour with d_k = 0 has no    */
/* interpolatory connection and is lumped into at as a_ik (its weight terms  */
/* are skipped); w_ij = -(num / at).  An empty Chat_i gives an empty row;   */
/* at = 0 fails the set-up (OR_ERR_SETUP).  Scalar problems only (bs = 1).   */
/* ------------------------------------------------------------------ */
static double abar(double akl) { return akl < 0.0 ? akl : 0.0; } /* a_kk > 0 on every level */

static int row_pos(const int *rp, const int *ci, int i, int j) {
  int lo = rp[i], hi = rp[i + 1] - 1;
  while (lo <= hi) {
    int mid = (lo + hi) / 2;
    if (ci[mid] == j) return mid;
    if (ci[mid] < j) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

static int in_sorted(const int *set, int m, int j) {
  int lo = 0, hi = m - 1;
  while (lo <= hi) {
    int mid = (lo + hi) / 2;
    if (set[mid] == j) return 1;
    if (set[mid] < j) lo = mid + 1;
    else hi = mid - 1;
  }
  return 0;
}

static int ext_interp(int n, const int *rp, const int *ci, const double *a, const unsigned char *S,
                      const signed char *cf, int *cidx, int *nc_out, int *Prp, int *Pci, double *Pv, long long cap) {
  int nc = 0;
  for (int i = 0; i < n; ++i) cidx[i] = cf[i] ? nc++ : -1;
  *nc_out = nc;
  int maxrow = 0;
  for (int i = 0; i < n; ++i)
    if (rp[i + 1] - rp[i] > maxrow) maxrow = rp[i + 1] - rp[i];
  size_t candcap = (size_t)maxrow * (size_t)maxrow + 1;
  int *cand = (int *)malloc(candcap * sizeof(int));
  double *d = (double *)malloc(((size_t)maxrow + 1) * sizeof(double));
  if (!cand || !d) {
    free(cand); free(d);
    return OR_ERR_MEM;
  }
  long long pos = 0;
  Prp[0] = 0;
  for (int i = 0; i < n; ++i) {
    if (cf[i]) {
      if (pos + 1 > cap) { free(cand); free(d); return OR_ERR_MEM; }
      Pci[pos] = cidx[i];
      Pv[pos] = 1.0;
      ++pos;
      Prp[i + 1] = (int)pos;
      continue;
    }
    /* Chat_i: strong C neighbours of i and of its strong F neighbours */
    int m = 0;
    double aii = 0.0;
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      int k = ci[p];
      if (k == i) aii = a[p];
      if (k == i || !S[p]) continue;
      if (cf[k]) {
        cand[m++] = k;
      } else {
        for (int q = rp[k]; q < rp[k + 1]; ++q)
          if (S[q] && ci[q] != k && cf[ci[q]]) cand[m++] = ci[q];
      }
    }
    qsort(cand, (size_t)m, sizeof(int), cmp_int);
    int u = 0;
    for (int t = 0; t < m; ++t)
      if (u == 0 || cand[t] != cand[u - 1]) cand[u++] = cand[t];
    m = u;
    if (m == 0) {
      Prp[i + 1] = (int)pos;
      continue;
    }
    /* d_k for every strong F neighbour k (indexed by its position in row i) */
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      int k = ci[p];
      d[p - rp[i]] = 0.0;
      if (k == i || !S[p] || cf[k]) continue;
      double dk = 0.0;
      for (int q = rp[k]; q < rp[k + 1]; ++q) {
        int l = ci[q];
        double ab = abar(a[q]);
        if (l == k || ab == 0.0) continue;
        if (l == i || in_sorted(cand, m, l)) dk += ab;
      }
      d[p - rp[i]] = dk;
    }
    /* at = a_ii + lumped weak couplings + the F_i^S terms toward i */
    double at = aii;
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      int k = ci[p];
      if (k == i) continue;
      if (S[p] && !cf[k]) {
        double dk = d[p - rp[i]];
        if (dk != 0.0) {
          int q = row_pos(rp, ci, k, i);
          double ab = q >= 0 ? abar(a[q]) : 0.0;
          if (ab != 0.0) at += (a[p] * ab) / dk;
        } else {
          at += a[p];
        }
      } else if (!S[p] && !(cf[k] && in_sorted(cand, m, k))) {
        at += a[p];
      }
    }
    if (at == 0.0) {
      free(cand); free(d);
      return OR_ERR_SETUP;
    }
    if (pos + m > cap) { free(cand); free(d); return OR_ERR_MEM; }
    for (int t = 0; t < m; ++t) {
      int j = cand[t];
      int qj = row_pos(rp, ci, i, j);
      double num = qj >= 0 ? a[qj] : 0.0;
      for (int p = rp[i]; p < rp[i + 1]; ++p) {
        int k = ci[p];
        if (k == i || !S[p] || cf[k]) continue;
        double dk = d[p - rp[i]];
        if (dk == 0.0) continue;
        int q = row_pos(rp, ci, k, j);
        double ab = q >= 0 ? abar(a[q]) : 0.0;
        if (ab != 0.0) num += (a[p] * ab) / dk;
      }
      Pci[pos] = cidx[j];
      Pv[pos] = -(num / at);
      ++pos;
    }
    Prp[i + 1] = (int)pos;
  }
  free(cand); free(d);
  return OR_OK;
}

int or_ext_interp(int n, const int *rp, const int *ci, const double *a, const unsigned char *S,
                  const signed char *cf, int *cidx, int *nc_out, int *Prp, int *Pci, double *Pv, long long cap) {
  return ext_interp(n, rp, ci, a, S, cf, cidx, nc_out, Prp, Pci, Pv, cap);
}

/* R = P^T, rows of R listing fine indices in ascending order. */
static int transpose(const or_csr *P, int ncols, or_csr *R) {
  if (csr_alloc(R, ncols, P->nnz)) return OR_ERR_MEM;
  for (int p = 0; p < P->nnz; ++p) R->rp[P->ci[p] + 1]++;
  for (int I = 0; I < ncols; ++I) R->rp[I + 1] += R->rp[I];
  int *fill = (int *)malloc(((size_t)ncols + 1) * sizeof(int));
  if (!fill) return OR_ERR_MEM;
  memcpy(fill, R->rp, (size_t)ncols * sizeof(int));
  for (int i = 0; i < P->n; ++i)
    for (int p = P->rp[i]; p < P->rp[i + 1]; ++p) {
      int q = fill[P->ci[p]]++;
      R->ci[q] = i;
      R->v[q] = P->v[p];
    }
  free(fill);
  return OR_OK;
}

static int cmp_int(const void *x, const void *y) {
  int a = *(const int *)x, b = *(const int *)y;
  return (a > b) - (a < b);
}

/* C = X Y with a dense accumulator: row i of C sums, over k ascending in   */
/* row i of X, the products x_ik * Y_kJ; each J's terms arrive in k order. */
/* Every structurally produced entry is kept (no dropping of zeros).       */
static int spgemm(const or_csr *X, const or_csr *Y, int ncols, or_csr *C) {
  double *acc = (double *)calloc((size_t)ncols + 1, sizeof(double));
  int *mark = (int *)malloc(((size_t)ncols + 1) * sizeof(int));
  int *list = (int *)malloc(((size_t)ncols + 1) * sizeof(int));
  if (!acc || !mark || !list) return OR_ERR_MEM;
  for (int J = 0; J < ncols; ++J) mark[J] = -1;
  /* pass 1: count */
  long long total = 0;
  for (int i = 0; i < X->n; ++i) {
    int cnt = 0;
    for (int p = X->rp[i]; p < X->rp[i + 1]; ++p) {
      int k = X->ci[p];
      for (int q = Y->rp[k]; q < Y->rp[k + 1]; ++q) {
        int J = Y->ci[q];
        if (mark[J] != i) {
          mark[J] = i;
          ++cnt;
        }
      }
    }
    total += cnt;
  }
  if (total >= 2147483647LL) return OR_ERR_MEM;
  if (csr_alloc(C, X->n, (int)total)) return OR_ERR_MEM;
  for (int J = 0; J < ncols; ++J) mark[J] = -1;
  /* pass 2: accumulate in canonical order, emit sorted */
  int pos = 0;
  for (int i = 0; i < X->n; ++i) {
    int cnt = 0;
    for (int p = X->rp[i]; p < X->rp[i + 1]; ++p) {
      int k = X->ci[p];
      double x = X->v[p];
      for (int q = Y->rp[k]; q < Y->rp[k + 1]; ++q) {
        int J = Y->ci[q];
        if (mark[J] != i) {
          mark[J] = i;
          acc[J] = 0.0;
          list[cnt++] = J;
        }
        double prod = x * Y->v[q];
        acc[J] = acc[J] + prod;
      }
    }
    qsort(list, (size_t)cnt, sizeof(int), cmp_int);
    for (int t = 0; t < cnt; ++t) {
      C->ci[pos] = list[t];
      C->v[pos] = acc[list[t]];
      ++pos;
    }
    C->rp[i + 1] = pos;
  }
  free(acc); free(mark); free(list);
  return OR_OK;
}

/* Galerkin coarse operator A_c = R (A P), R = P^T (Eq. AcDef). */
int or_galerkin(int n, const int *Arp, const int *Aci, const double *Av, int nc, const int *Prp,
                const int *Pci, const double *Pv, int *nnz_out, int **rp_out, int **ci_out,
                double **v_out) {
  or_csr A = {n, Arp[n], (int *)Arp, (int *)Aci, (double *)Av};
  or_csr P = {n, Prp[n], (int *)Prp, (int *)Pci, (double *)Pv};
  or_csr R, AP, Ac;
  memset(&R, 0, sizeof R); memset(&AP, 0, sizeof AP); memset(&Ac, 0, sizeof Ac);
  int st = transpose(&P, nc, &R);
  if (!st) st = spgemm(&A, &P, nc, &AP);
  if (!st) st = spgemm(&R, &AP, nc, &Ac);
  csr_free(&R);
  csr_free(&AP);
  if (st) {
    csr_free(&Ac);
    return st;
  }
  *nnz_out = Ac.nnz;
  *rp_out = Ac.rp;
  *ci_out = Ac.ci;
  *v_out = Ac.v;
  return OR_OK;
}

void or_free_array(void *p) { free(p); }

/* ------------------------------------------------------------------ */
/* Dense Cholesky A = L L^T (Algorithm 1, last level) and its solve.      */
/* ------------------------------------------------------------------ */
int or_cholesky(int n, double *M) {
  for (int j = 0; j < n; ++j) {
    double d = M[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= M[(size_t)j * n + k] * M[(size_t)j * n + k];
    if (!(d > 0.0)) return OR_ERR_NOT_SPD;
    double ljj = sqrt(d);
    M[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double s = M[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) s -= M[(size_t)i * n + k] * M[(size_t)j * n + k];
      M[(size_t)i * n + j] = s / ljj;
    }
    for (int i = 0; i < j; ++i) M[(size_t)i * n + j] = 0.0;
  }
  return OR_OK;
}

void or_cholesky_solve(int n, const double *L, const double *y, double *z) {
  for (int i = 0; i < n; ++i) {
    double s = y[i];
    for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * z[k];
    z[i] = s / L[(size_t)i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = z[i];
    for (int k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * z[k];
    z[i] = s / L[(size_t)i * n + i];
  }
}

/* y = A x */
void or_spmv(int n, const int *rp, const int *ci, const double *a, const double *x, double *y) {
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int p = rp[i]; p < rp[i + 1]; ++p) s += a[p] * x[ci[p]];
    y[i] = s;
  }
}

/* One damped-Jacobi step s <- s + omega D^{-1} (y - A s)  (Eq. smoother, M = D). */
void or_jacobi_sweep(int n, const int *rp, const int *ci, const double *a, double omega, const double *y,
                     double *s) {
  double *t = (double *)malloc((size_t)n * sizeof(double));
  for (int i = 0; i < n; ++i) {
    double r = y[i], d = 0.0;
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      r -= a[p] * s[ci[p]];
      if (ci[p] == i) d = a[p];
    }
    t[i] = s[i] + omega * r / d;
  }
  memcpy(s, t, (size_t)n * sizeof(double));
  free(t);
}

/* ------------------------------------------------------------------ */
/* Factored sparse approximate inverse (Eq. smo: M^{-1} = G^T G, G lower  */
/* triangular).  The paper's aFSAI grows the pattern of G adaptively      */
/* (cited, not described); the reading taken here is the static FSAI of   */
/* Kolotilina & Yeremin on the pattern of the lower triangle of A:        */
/* for row i, P_i = { j <= i : a_ij stored } (ascending, last = i),        */
/*   solve A[P_i, P_i] gt = e_last (dense Cholesky of the principal        */
/*   submatrix, which is SPD when A is), then g_i = gt / sqrt(gt_last),   */
/* so that (G A G^T)_ii = 1.  Grp[n+1], Gci / Gv with room for nnz(A).    */
/* ------------------------------------------------------------------ */
static double csr_entry(const int *rp, const int *ci, const double *a, int i, int j) {
  for (int p = rp[i]; p < rp[i + 1]; ++p)
    if (ci[p] == j) return a[p];
  return 0.0;
}

int or_fsai(int n, const int *rp, const int *ci, const double *a, int *Grp, int *Gci, double *Gv) {
  int mmax = 0;
  for (int i = 0; i < n; ++i) {
    int m = 0;
    for (int p = rp[i]; p < rp[i + 1]; ++p) m += (ci[p] <= i);
    if (m > mmax) mmax = m;
  }
  int *P = (int *)malloc(((size_t)mmax + 1) * sizeof(int));
  double *M = (double *)malloc(((size_t)mmax * mmax + 1) * sizeof(double));
  double *e = (double *)malloc(((size_t)mmax + 1) * sizeof(double));
  double *g = (double *)malloc(((size_t)mmax + 1) * sizeof(double));
  if (!P || !M || !e || !g) {
    free(P); free(M); free(e); free(g);
    return OR_ERR_MEM;
  }
  int pos = 0, st = OR_OK;
  Grp[0] = 0;
  for (int i = 0; i < n && !st; ++i) {
    int m = 0;
    for (int p = rp[i]; p < rp[i + 1]; ++p)
      if (ci[p] <= i) P[m++] = ci[p];
    if (m == 0 || P[m - 1] != i) {
      st = OR_ERR_ARG; /* no diagonal */
      break;
    }
    for (int r = 0; r < m; ++r)
      for (int c = 0; c < m; ++c) M[(size_t)r * m + c] = csr_entry(rp, ci, a, P[r], P[c]);
    if (or_cholesky(m, M)) {
      st = OR_ERR_NOT_SPD;
      break;
    }
    for (int r = 0; r < m; ++r) e[r] = (r == m - 1) ? 1.0 : 0.0;
    or_cholesky_solve(m, M, e, g);
    if (!(g[m - 1] > 0.0)) {
      st = OR_ERR_NOT_SPD;
      break;
    }
    double scale = sqrt(g[m - 1]);
    for (int r = 0; r < m; ++r) {
      Gci[pos] = P[r];
      Gv[pos] = g[r] / scale;
      ++pos;
    }
    Grp[i + 1] = pos;
  }
  free(P); free(M); free(e); free(g);
  return st;
}

/* One FSAI smoothing step s <- s + omega G^T G (y - A s)  (Eq. smoother with */
/* M^{-1} = G^T G).  G^T u is formed by scattering each row of G.            */
void or_fsai_sweep(int n, const int *rp, const int *ci, const double *a, const int *Grp, const int *Gci,
                   const double *Gv, double omega, const double *y, double *s) {
  double *r = (double *)malloc((size_t)n * sizeof(double));
  double *u = (double *)malloc((size_t)n * sizeof(double));
  double *w = (double *)calloc((size_t)n, sizeof(double));
  for (int i = 0; i < n; ++i) {
    double t = y[i];
    for (int p = rp[i]; p < rp[i + 1]; ++p) t -= a[p] * s[ci[p]];
    r[i] = t;
  }
  for (int i = 0; i < n; ++i) {
    double t = 0.0;
    for (int p = Grp[i]; p < Grp[i + 1]; ++p) t += Gv[p] * r[Gci[p]];
    u[i] = t;
  }
  for (int i = 0; i < n; ++i)
    for (int p = Grp[i]; p < Grp[i + 1]; ++p) w[Gci[p]] += Gv[p] * u[i];
  for (int i = 0; i < n; ++i) s[i] += omega * w[i];
  free(r); free(u); free(w);
}

/* ------------------------------------------------------------------ */
/* Algorithm 1: AMG set-up.                                               */
/* Stop on: n_k <= max_coarse, level max_levels-1 reached, or a stalled   */
/* coarsening (n_{k+1} == 0 or n_{k+1} > 0.9 n_k).  The last level is      */
/* factorised densely (error if it has more than 4096 rows).              */
/* ------------------------------------------------------------------ */
void or_free(or_hier *h);

int or_setup_ex(int n, const int *rp, const int *ci, const double *a, double theta, uint64_t seed,
                int max_coarse, int max_levels, double omega, int nu1, int nu2, int bs, int smoother, int interp,
                or_hier **out);

int or_setup(int n, const int *rp, const int *ci, const double *a, double theta, uint64_t seed,
             int max_coarse, int max_levels, double omega, int nu1, int nu2, or_hier **out) {
  return or_setup_ex(n, rp, ci, a, theta, seed, max_coarse, max_levels, omega, nu1, nu2, 1, 0, 0, out);
}

int or_setup_bs(int n, const int *rp, const int *ci, const double *a, double theta, uint64_t seed,
                int max_coarse, int max_levels, double omega, int nu1, int nu2, int bs, or_hier **out) {
  return or_setup_ex(n, rp, ci, a, theta, seed, max_coarse, max_levels, omega, nu1, nu2, bs, 0, 0, out);
}

/* Algorithm 1.  bs = 1: scalar strength and PMIS on the unknowns.  bs > 1  */
/* (systems, node-major unknowns): nodal block strength, PMIS on the node   */
/* graph (the measure counter runs over node indices), every unknown of a   */
/* node takes the node's C/F label, and unknown-wise direct interpolation.  */
/* smoother: 0 damped Jacobi, 1 FSAI (G formed on every level but the last). */
/* interp: 0 direct interpolation, 1 extended+i (bs = 1).                   */
int or_setup_ex(int n, const int *rp, const int *ci, const double *a, double theta, uint64_t seed,
                int max_coarse, int max_levels, double omega, int nu1, int nu2, int bs, int smoother, int interp,
                or_hier **out) {
  *out = NULL;
  if (!(theta > 0.0 && theta <= 1.0) || max_levels < 1 || max_levels > OR_MAX_LEVELS || nu1 < 0 ||
      nu2 < 0 || max_coarse < 1 || bs < 1 || n % bs || smoother < 0 || smoother > 1 || interp < 0 ||
      interp > 1 || (interp == 1 && bs != 1))
    return OR_ERR_ARG;
  int st = or_check_csr(n, rp, ci, a);
  if (st) return st;
  or_hier *h = (or_hier *)calloc(1, sizeof(or_hier));
  if (!h) return OR_ERR_MEM;
  h->omega = omega;
  h->nu1 = nu1;
  h->nu2 = nu2;
  h->smoother = smoother;
  if (csr_alloc(&h->A[0], n, rp[n])) {
    or_free(h);
    return OR_ERR_MEM;
  }
  memcpy(h->A[0].rp, rp, ((size_t)n + 1) * sizeof(int));
  memcpy(h->A[0].ci, ci, (size_t)rp[n] * sizeof(int));
  memcpy(h->A[0].v, a, (size_t)rp[n] * sizeof(double));

  int k = 0;
  for (;;) {
    or_csr *A = &h->A[k];
    int nk = A->n;
    h->wr[k] = (double *)calloc((size_t)nk, sizeof(double));
    h->wy[k] = (double *)calloc((size_t)nk, sizeof(double));
    h->wz[k] = (double *)calloc((size_t)nk, sizeof(double));
    h->ws[k] = (double *)calloc((size_t)nk, sizeof(double));
    int last = (nk <= max_coarse) || (k == max_levels - 1);
    if (!last) {
      h->S[k] = (unsigned char *)malloc((size_t)A->nnz + 1);
      h->cf[k] = (signed char *)malloc((size_t)nk);
      if (bs == 1) {
        or_strength(nk, A->rp, A->ci, A->v, theta, h->S[k]);
        st = or_pmis(nk, A->rp, A->ci, h->S[k], seed, k, h->cf[k]);
      } else {
        int nn = 0;
        int *Nrp = (int *)malloc(((size_t)nk / bs + 1) * sizeof(int));
        int *Nci = (int *)malloc(((size_t)A->nnz + 1) * sizeof(int));
        unsigned char *SN = (unsigned char *)malloc((size_t)A->nnz + 1);
        signed char *cfn = (signed char *)malloc((size_t)nk / bs + 1);
        st = (Nrp && Nci && SN && cfn) ? OR_OK : OR_ERR_MEM;
        if (!st) st = or_block_strength(nk, A->rp, A->ci, A->v, bs, theta, &nn, Nrp, Nci, SN, h->S[k]);
        if (!st) st = or_pmis(nn, Nrp, Nci, SN, seed, k, cfn);
        if (!st)
          for (int i = 0; i < nk; ++i) h->cf[k][i] = cfn[i / bs];
        free(Nrp); free(Nci); free(SN); free(cfn);
      }
      if (st) {
        or_free(h);
        return st;
      }
      int nc = 0;
      for (int i = 0; i < nk; ++i) nc += h->cf[k][i];
      if (nc == 0 || (double)nc > 0.9 * (double)nk) {
        last = 1; /* stalled coarsening: this level becomes the last one */
      } else {
        long long cap = (long long)A->nnz + nk;
        if (interp == 1) { /* |Chat_i| <= sum over the row's strong neighbours of their row lengths */
          cap = nk;
          for (int i = 0; i < nk; ++i)
            for (int p = A->rp[i]; p < A->rp[i + 1]; ++p) cap += A->rp[A->ci[p] + 1] - A->rp[A->ci[p]];
        }
        or_csr *P = &h->P[k];
        if (cap >= 2147483647LL || csr_alloc(P, nk, (int)cap)) {
          or_free(h);
          return OR_ERR_MEM;
        }
        int *cidx = (int *)malloc((size_t)nk * sizeof(int));
        int ncc = 0;
        if (interp == 1)
          st = ext_interp(nk, A->rp, A->ci, A->v, h->S[k], h->cf[k], cidx, &ncc, P->rp, P->ci, P->v, cap);
        else
          st = direct_interp(nk, A->rp, A->ci, A->v, h->S[k], h->cf[k], bs, cidx, &ncc, P->rp, P->ci, P->v, cap);
        free(cidx);
        if (st) {
          or_free(h);
          return st;
        }
        P->nnz = P->rp[nk];
        st = transpose(P, nc, &h->R[k]);
        or_csr AP;
        memset(&AP, 0, sizeof AP);
        if (!st) st = spgemm(A, P, nc, &AP);
        if (!st) st = spgemm(&h->R[k], &AP, nc, &h->A[k + 1]);
        csr_free(&AP);
        if (!st && smoother == 1) {
          or_csr *G = &h->G[k];
          st = csr_alloc(G, nk, A->nnz);
          if (!st) st = or_fsai(nk, A->rp, A->ci, A->v, G->rp, G->ci, G->v);
          if (!st) G->nnz = G->rp[nk];
        }
        if (st) {
          or_free(h);
          return st;
        }
        ++k;
        continue;
      }
    }
    /* last level: dense Cholesky */
    free(h->S[k]);
    h->S[k] = NULL;
    free(h->cf[k]);
    h->cf[k] = NULL;
    if (nk > OR_MAX_DENSE) {
      or_free(h);
      return OR_ERR_SETUP;
    }
    h->nL = nk;
    h->L = (double *)calloc((size_t)nk * nk, sizeof(double));
    for (int i = 0; i < nk; ++i)
      for (int p = A->rp[i]; p < A->rp[i + 1]; ++p) h->L[(size_t)i * nk + A->ci[p]] = A->v[p];
    st = or_cholesky(nk, h->L);
    if (st) {
      or_free(h);
      return st;
    }
    h->nlevels = k + 1;
    break;
  }
  *out = h;
  return OR_OK;
}

void or_free(or_hier *h) {
  if (!h) return;
  for (int k = 0; k < OR_MAX_LEVELS; ++k) {
    csr_free(&h->A[k]);
    csr_free(&h->P[k]);
    csr_free(&h->R[k]);
    csr_free(&h->G[k]);
    free(h->cf[k]);
    free(h->S[k]);
    free(h->wr[k]);
    free(h->wy[k]);
    free(h->wz[k]);
    free(h->ws[k]);
  }
  free(h->L);
  free(h);
}

int or_nlevels(const or_hier *h) { return h->nlevels; }

void or_level_info(const or_hier *h, int k, int *n, int *nnzA, int *nnzP) {
  *n = h->A[k].n;
  *nnzA = h->A[k].nnz;
  *nnzP = (k < h->nlevels - 1) ? h->P[k].nnz : 0;
}

void or_get_A(const or_hier *h, int k, int *rp, int *ci, double *v) {
  const or_csr *m = &h->A[k];
  memcpy(rp, m->rp, ((size_t)m->n + 1) * sizeof(int));
  memcpy(ci, m->ci, (size_t)m->nnz * sizeof(int));
  memcpy(v, m->v, (size_t)m->nnz * sizeof(double));
}

void or_get_P(const or_hier *h, int k, int *rp, int *ci, double *v) {
  const or_csr *m = &h->P[k];
  memcpy(rp, m->rp, ((size_t)m->n + 1) * sizeof(int));
  memcpy(ci, m->ci, (size_t)m->nnz * sizeof(int));
  memcpy(v, m->v, (size_t)m->nnz * sizeof(double));
}

int or_G_nnz(const or_hier *h, int k) { return (k < h->nlevels - 1 && h->smoother == 1) ? h->G[k].nnz : 0; }

void or_get_G(const or_hier *h, int k, int *rp, int *ci, double *v) {
  const or_csr *m = &h->G[k];
  memcpy(rp, m->rp, ((size_t)m->n + 1) * sizeof(int));
  memcpy(ci, m->ci, (size_t)m->nnz * sizeof(int));
  memcpy(v, m->v, (size_t)m->nnz * sizeof(double));
}

void or_get_cf(const or_hier *h, int k, signed char *cf) { memcpy(cf, h->cf[k], (size_t)h->A[k].n); }

void or_get_S(const or_hier *h, int k, unsigned char *S) { memcpy(S, h->S[k], (size_t)h->A[k].nnz); }

void or_complexities(const or_hier *h, double *cgd, double *cop) {
  double sn = 0.0, sz = 0.0;
  for (int k = 0; k < h->nlevels; ++k) {
    sn += h->A[k].n;
    sz += h->A[k].nnz;
  }
  *cgd = sn / h->A[0].n;
  *cop = sz / h->A[0].nnz;
}

/* ------------------------------------------------------------------ */
/* Algorithm 2: V-cycle z_k = B_k y_k.                                    */
/* ------------------------------------------------------------------ */
/* one smoothing step s <- s + omega M^{-1} (y - A s) on level k (Eq. smoother) */
static void smooth(or_hier *h, int k, const double *y, double *s) {
  const or_csr *A = &h->A[k];
  if (h->smoother == 1) {
    const or_csr *G = &h->G[k];
    or_fsai_sweep(A->n, A->rp, A->ci, A->v, G->rp, G->ci, G->v, h->omega, y, s);
  } else {
    or_jacobi_sweep(A->n, A->rp, A->ci, A->v, h->omega, y, s);
  }
}

static void vcycle(or_hier *h, int k, const double *y, double *z) {
  const or_csr *A = &h->A[k];
  int n = A->n;
  if (k == h->nlevels - 1) {
    or_cholesky_solve(n, h->L, y, z);
    return;
  }
  double *s = h->ws[k], *r = h->wr[k];
  /* nu1 smoothing steps on A s = y from s = 0 */
  for (int i = 0; i < n; ++i) s[i] = 0.0;
  for (int it = 0; it < h->nu1; ++it) smooth(h, k, y, s);
  /* residual r = y - A s */
  or_spmv(n, A->rp, A->ci, A->v, s, r);
  for (int i = 0; i < n; ++i) r[i] = y[i] - r[i];
  /* restriction r_{k+1} = P^T r */
  const or_csr *R = &h->R[k];
  double *yc = h->wy[k + 1], *dc = h->wz[k + 1];
  or_spmv(R->n, R->rp, R->ci, R->v, r, yc);
  vcycle(h, k + 1, yc, dc);
  /* prolongation d = P d_{k+1}; s <- s + d */
  const or_csr *P = &h->P[k];
  or_spmv(n, P->rp, P->ci, P->v, dc, r);
  for (int i = 0; i < n; ++i) s[i] += r[i];
  /* nu2 smoothing steps from z = s */
  for (int i = 0; i < n; ++i) z[i] = s[i];
  for (int it = 0; it < h->nu2; ++it) smooth(h, k, y, z);
}

void or_vcycle(or_hier *h, const double *y, double *z) {
  double *y0 = (double *)malloc((size_t)h->A[0].n * sizeof(double));
  memcpy(y0, y, (size_t)h->A[0].n * sizeof(double));
  vcycle(h, 0, y0, z);
  free(y0);
}

static double dot(int n, const double *x, const double *y) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += x[i] * y[i];
  return s;
}

/* ------------------------------------------------------------------ */
/* PCG (Sec. 3.1 solver; stopping rule of Sec. 4).  x holds x0 on entry.  */
/* precond: 0 = identity, 1 = one V-cycle.  flexible: beta from           */
/* (z_{k+1}, r_{k+1} - r_k) / (z_k, r_k) instead of (z_{k+1}, r_{k+1}) /  */
/* (z_k, r_k).  hist[0..iters] receives ||r_k||_2; xhist (may be NULL)    */
/* receives x after every iteration (row it-1 of an maxit x n array).     */
/* ------------------------------------------------------------------ */
int or_pcg(or_hier *h, const double *b, double *x, double rtol, int maxit, int flexible, int precond,
           int *iters, double *hist, double *xhist) {
  const or_csr *A = &h->A[0];
  int n = A->n;
  double *r = (double *)malloc((size_t)n * sizeof(double));
  double *z = (double *)malloc((size_t)n * sizeof(double));
  double *p = (double *)malloc((size_t)n * sizeof(double));
  double *q = (double *)malloc((size_t)n * sizeof(double));
  double *rold = (double *)malloc((size_t)n * sizeof(double));
  int st = OR_ERR_NO_CONVERGENCE;
  or_spmv(n, A->rp, A->ci, A->v, x, q);
  for (int i = 0; i < n; ++i) r[i] = b[i] - q[i];
  double bnorm = sqrt(dot(n, b, b));
  double res = sqrt(dot(n, r, r));
  if (hist) hist[0] = res;
  *iters = 0;
  if (res < rtol * bnorm || bnorm == 0.0) {
    st = OR_OK;
    goto done;
  }
  if (precond) or_vcycle(h, r, z);
  else memcpy(z, r, (size_t)n * sizeof(double));
  memcpy(p, z, (size_t)n * sizeof(double));
  double rho = dot(n, r, z);
  for (int it = 1; it <= maxit; ++it) {
    or_spmv(n, A->rp, A->ci, A->v, p, q);
    double pq = dot(n, p, q);
    if (!(pq > 0.0)) {
      st = OR_ERR_BREAKDOWN;
      break;
    }
    double alpha = rho / pq;
    memcpy(rold, r, (size_t)n * sizeof(double));
    for (int i = 0; i < n; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * q[i];
    }
    res = sqrt(dot(n, r, r));
    *iters = it;
    if (hist) hist[it] = res;
    if (xhist) memcpy(xhist + (size_t)(it - 1) * n, x, (size_t)n * sizeof(double));
    if (res < rtol * bnorm) {
      st = OR_OK;
      break;
    }
    if (precond) or_vcycle(h, r, z);
    else memcpy(z, r, (size_t)n * sizeof(double));
    double rho_new = dot(n, r, z), beta;
    if (flexible) {
      for (int i = 0; i < n; ++i) rold[i] = r[i] - rold[i];
      beta = dot(n, z, rold) / rho;
    } else {
      beta = rho_new / rho;
    }
    rho = rho_new;
    for (int i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
  }
done:
  free(r); free(z); free(p); free(q); free(rold);
  return st;
}
