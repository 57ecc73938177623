/*
 * CPU oracle for the feasible reduced-space OPF hot path (arXiv 2110.02590).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the library.  Plain FP64 C, written
 * for readability: it computes the power-flow solution, the reduced gradient
 * and the reduced Hessian from their definitions, with no blocking or fusion.
 *
 *   power flow         Newton-Raphson x <- x - (G_x)^{-1} g          eq. projection:newtonraphson
 *   reduced gradient   G_x^T lam = -(d_x F)^T, grad = d_u F + lam^T G_u   Prop. 1
 *   reduced Hessian    G_x z = -G_u w ; G_x^T psi = -(l_xu w + l_xx z) ;
 *                      H w = l_uu w + l_ux z + G_u^T psi                 Prop. 2
 *   AL functional      sigma_f f + y^T D_c (c - s) + rho/2 |D_c (c - s)|^2   Sec. IV-A
 *
 * The second derivatives of l = F + lam^T g are assembled explicitly as a
 * sparse matrix over the bus variables (v_i, theta_i, p_k) from the polar
 * branch-flow formulas.  An independent brute force (orc_bruteforce) takes
 * them instead from hyper-dual numbers (Fike & Alonso 2011) applied to the
 * complex-voltage form S = V conj(Y V) with a dense bus admittance matrix.
 *
 * Sparse LU: exact minimum degree on the bus graph (node weight = number of
 * state variables of the bus, degree = sum of neighbour weights, ties broken
 * by smallest bus id), variables of a bus consecutive (theta before v), LU
 * without pivoting on the filled pattern, row by row.
 */
#include "opf_oracle.h"

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { BUS_REF = 0, BUS_PV = 1, BUS_PQ = 2 };
enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOMEM = -2, ORC_ENOCONV = -3, ORC_ESINGULAR = -4,
       ORC_ENOTPD = -5 };

struct orc_net {
  int nb, nl, ng, ref, npv, npq, nx, nu, m;
  double *pd, *qd, *vmin, *vmax;
  int *f, *t;
  double *rate;
  double *Gff, *Bff, *Gft, *Bft, *Gtf, *Btf, *Gtt, *Btt;
  int* gbus;
  double *c2, *c1, *c0, *pmin, *pmax, *qmin, *qmax;
  int* type;     /* per bus */
  int* gen_at;   /* per bus: generator index or -1 */
  int *pv, *pq;  /* bus lists */
  int* pvpos;    /* per bus: position in pv list or -1 */
  int *xth, *xv; /* per bus: x index of theta / v, or -1 */
  int *zv, *zth; /* per bus: index in z = (x, u) of v / theta, or -1 */
  /* symbolic */
  int sym_done;
  int nsb;       /* number of state buses */
  int* bus_order;
  int *perm, *iperm; /* perm[new] = old x index */
  int *rp, *ci, *dp; /* full filled pattern, row-wise, new indices, sorted */
  int nnz;
  int *lev_f, *lev_b;
};

/* ------------------------------------------------------------------ utils */

static void* xcalloc(size_t n, size_t sz) {
  if (n == 0) n = 1;
  return calloc(n, sz);
}

static double* dup_d(const double* a, int n) {
  double* r = (double*)xcalloc((size_t)n, sizeof(double));
  if (r && a) memcpy(r, a, sizeof(double) * (size_t)n);
  return r;
}

static int* dup_i(const int* a, int n) {
  int* r = (int*)xcalloc((size_t)n, sizeof(int));
  if (r && a) memcpy(r, a, sizeof(int) * (size_t)n);
  return r;
}

/* COO accumulator and CSR with duplicate summation. */
typedef struct {
  int len, cap;
  int *r, *c;
  double* v;
} coo_t;

typedef struct {
  int nr, nc;
  int *rp, *ci;
  double* v;
} csr_t;

static void coo_add(coo_t* a, int r, int c, double v) {
  if (r < 0 || c < 0) return;
  if (a->len == a->cap) {
    int nc = a->cap ? 2 * a->cap : 1024;
    a->r = (int*)realloc(a->r, sizeof(int) * (size_t)nc);
    a->c = (int*)realloc(a->c, sizeof(int) * (size_t)nc);
    a->v = (double*)realloc(a->v, sizeof(double) * (size_t)nc);
    a->cap = nc;
  }
  a->r[a->len] = r;
  a->c[a->len] = c;
  a->v[a->len] = v;
  a->len++;
}

static void coo_free(coo_t* a) {
  free(a->r);
  free(a->c);
  free(a->v);
  memset(a, 0, sizeof(*a));
}

/* Build CSR; duplicates are summed in insertion order. */
static csr_t coo_to_csr(const coo_t* a, int nr, int nc) {
  csr_t m;
  m.nr = nr;
  m.nc = nc;
  int* cnt = (int*)xcalloc((size_t)nr + 1, sizeof(int));
  for (int k = 0; k < a->len; k++) cnt[a->r[k] + 1]++;
  for (int i = 0; i < nr; i++) cnt[i + 1] += cnt[i];
  int* pos = (int*)xcalloc((size_t)nr + 1, sizeof(int));
  memcpy(pos, cnt, sizeof(int) * ((size_t)nr + 1));
  int* tc = (int*)xcalloc((size_t)a->len, sizeof(int));
  double* tv = (double*)xcalloc((size_t)a->len, sizeof(double));
  for (int k = 0; k < a->len; k++) {
    int p = pos[a->r[k]]++;
    tc[p] = a->c[k];
    tv[p] = a->v[k];
  }
  /* per row: insertion sort by column, then merge duplicates */
  m.rp = (int*)xcalloc((size_t)nr + 1, sizeof(int));
  m.ci = (int*)xcalloc((size_t)a->len, sizeof(int));
  m.v = (double*)xcalloc((size_t)a->len, sizeof(double));
  int out = 0;
  for (int i = 0; i < nr; i++) {
    int b = cnt[i], e = cnt[i + 1];
    for (int p = b + 1; p < e; p++) {
      int kc = tc[p];
      double kv = tv[p];
      int q = p - 1;
      while (q >= b && tc[q] > kc) {
        tc[q + 1] = tc[q];
        tv[q + 1] = tv[q];
        q--;
      }
      tc[q + 1] = kc;
      tv[q + 1] = kv;
    }
    m.rp[i] = out;
    for (int p = b; p < e; p++) {
      if (out > m.rp[i] && m.ci[out - 1] == tc[p]) {
        m.v[out - 1] += tv[p];
      } else {
        m.ci[out] = tc[p];
        m.v[out] = tv[p];
        out++;
      }
    }
  }
  m.rp[nr] = out;
  free(cnt);
  free(pos);
  free(tc);
  free(tv);
  return m;
}

static void csr_free(csr_t* m) {
  free(m->rp);
  free(m->ci);
  free(m->v);
  memset(m, 0, sizeof(*m));
}

/* y = A x (y has nr entries) */
static void csr_mv(const csr_t* A, const double* x, double* y) {
  for (int i = 0; i < A->nr; i++) {
    double s = 0.0;
    for (int p = A->rp[i]; p < A->rp[i + 1]; p++) s += A->v[p] * x[A->ci[p]];
    y[i] = s;
  }
}

/* y = A^T x (y has nc entries) */
static void csr_mtv(const csr_t* A, const double* x, double* y) {
  for (int j = 0; j < A->nc; j++) y[j] = 0.0;
  for (int i = 0; i < A->nr; i++)
    for (int p = A->rp[i]; p < A->rp[i + 1]; p++) y[A->ci[p]] += A->v[p] * x[i];
}

/* ------------------------------------------------------------- network */

orc_net* orc_net_new(int nb, int nl, int ng, int ref, const double* pd, const double* qd,
                     const double* vmin, const double* vmax, const int* f, const int* t,
                     const double* r, const double* x, const double* b, const double* tap,
                     const double* rate, const int* gbus, const double* c2, const double* c1,
                     const double* c0, const double* pmin, const double* pmax,
                     const double* qmin, const double* qmax) {
  if (nb < 2 || nl < 1 || ng < 1 || ref < 0 || ref >= nb) return NULL;
  orc_net* n = (orc_net*)xcalloc(1, sizeof(orc_net));
  n->nb = nb;
  n->nl = nl;
  n->ng = ng;
  n->ref = ref;
  n->pd = dup_d(pd, nb);
  n->qd = dup_d(qd, nb);
  n->vmin = dup_d(vmin, nb);
  n->vmax = dup_d(vmax, nb);
  n->f = dup_i(f, nl);
  n->t = dup_i(t, nl);
  n->rate = dup_d(rate, nl);
  n->gbus = dup_i(gbus, ng);
  n->c2 = dup_d(c2, ng);
  n->c1 = dup_d(c1, ng);
  n->c0 = dup_d(c0, ng);
  n->pmin = dup_d(pmin, ng);
  n->pmax = dup_d(pmax, ng);
  n->qmin = dup_d(qmin, ng);
  n->qmax = dup_d(qmax, ng);
  for (int l = 0; l < nl; l++) {
    if (f[l] < 0 || f[l] >= nb || t[l] < 0 || t[l] >= nb || f[l] == t[l]) {
      orc_net_free(n);
      return NULL;
    }
  }
  /* branch pi-model: series y = 1/(r + jx), tap on the from side, charging b/2 per end */
  n->Gff = (double*)xcalloc((size_t)nl, sizeof(double));
  n->Bff = (double*)xcalloc((size_t)nl, sizeof(double));
  n->Gft = (double*)xcalloc((size_t)nl, sizeof(double));
  n->Bft = (double*)xcalloc((size_t)nl, sizeof(double));
  n->Gtf = (double*)xcalloc((size_t)nl, sizeof(double));
  n->Btf = (double*)xcalloc((size_t)nl, sizeof(double));
  n->Gtt = (double*)xcalloc((size_t)nl, sizeof(double));
  n->Btt = (double*)xcalloc((size_t)nl, sizeof(double));
  for (int l = 0; l < nl; l++) {
    double den = r[l] * r[l] + x[l] * x[l];
    double gs = r[l] / den, bs = -x[l] / den;
    double tau = tap[l];
    n->Gff[l] = gs / (tau * tau);
    n->Bff[l] = (bs + 0.5 * b[l]) / (tau * tau);
    n->Gft[l] = -gs / tau;
    n->Bft[l] = -bs / tau;
    n->Gtf[l] = -gs / tau;
    n->Btf[l] = -bs / tau;
    n->Gtt[l] = gs;
    n->Btt[l] = bs + 0.5 * b[l];
  }
  n->type = (int*)xcalloc((size_t)nb, sizeof(int));
  n->gen_at = (int*)xcalloc((size_t)nb, sizeof(int));
  for (int i = 0; i < nb; i++) {
    n->type[i] = BUS_PQ;
    n->gen_at[i] = -1;
  }
  for (int g = 0; g < ng; g++) {
    int bus = gbus[g];
    if (bus < 0 || bus >= nb || n->gen_at[bus] >= 0) {
      orc_net_free(n);
      return NULL;
    }
    n->gen_at[bus] = g;
    n->type[bus] = BUS_PV;
  }
  if (n->gen_at[ref] < 0) {
    orc_net_free(n);
    return NULL;
  }
  n->type[ref] = BUS_REF;
  n->pv = (int*)xcalloc((size_t)nb, sizeof(int));
  n->pq = (int*)xcalloc((size_t)nb, sizeof(int));
  n->pvpos = (int*)xcalloc((size_t)nb, sizeof(int));
  n->npv = n->npq = 0;
  for (int i = 0; i < nb; i++) {
    n->pvpos[i] = -1;
    if (n->type[i] == BUS_PV) {
      n->pvpos[i] = n->npv;
      n->pv[n->npv++] = i;
    } else if (n->type[i] == BUS_PQ) {
      n->pq[n->npq++] = i;
    }
  }
  n->nx = n->npv + 2 * n->npq;
  n->nu = 1 + 2 * n->npv;
  n->m = 2 * nl + n->npq + n->npv + 2;
  n->xth = (int*)xcalloc((size_t)nb, sizeof(int));
  n->xv = (int*)xcalloc((size_t)nb, sizeof(int));
  n->zv = (int*)xcalloc((size_t)nb, sizeof(int));
  n->zth = (int*)xcalloc((size_t)nb, sizeof(int));
  for (int i = 0; i < nb; i++) n->xth[i] = n->xv[i] = -1;
  for (int k = 0; k < n->npv; k++) n->xth[n->pv[k]] = k;
  for (int k = 0; k < n->npq; k++) {
    n->xth[n->pq[k]] = n->npv + k;
    n->xv[n->pq[k]] = n->npv + n->npq + k;
  }
  for (int i = 0; i < nb; i++) {
    n->zth[i] = n->xth[i];
    if (n->type[i] == BUS_PQ)
      n->zv[i] = n->xv[i];
    else if (n->type[i] == BUS_REF)
      n->zv[i] = n->nx + 0;
    else
      n->zv[i] = n->nx + 1 + n->pvpos[i];
  }
  return n;
}

void orc_net_free(orc_net* n) {
  if (!n) return;
  void* ptrs[] = {n->pd,   n->qd,   n->vmin, n->vmax, n->f,     n->t,    n->rate,   n->Gff,
                  n->Bff,  n->Gft,  n->Bft,  n->Gtf,  n->Btf,   n->Gtt,  n->Btt,    n->gbus,
                  n->c2,   n->c1,   n->c0,   n->pmin, n->pmax,  n->qmin, n->qmax,   n->type,
                  n->gen_at, n->pv, n->pq,   n->pvpos, n->xth,  n->xv,   n->zv,     n->zth,
                  n->bus_order, n->perm, n->iperm, n->rp, n->ci, n->dp, n->lev_f, n->lev_b};
  for (size_t k = 0; k < sizeof(ptrs) / sizeof(ptrs[0]); k++) free(ptrs[k]);
  free(n);
}

int orc_dims(const orc_net* n, int* nx, int* nu, int* m, int* npv, int* npq) {
  if (!n) return ORC_EINVAL;
  if (nx) *nx = n->nx;
  if (nu) *nu = n->nu;
  if (m) *m = n->m;
  if (npv) *npv = n->npv;
  if (npq) *npq = n->npq;
  return ORC_OK;
}

/* --------------------------------------------------------- symbolic */

/* Exact minimum degree on the bus graph of the state buses with bitset rows. */
static int symbolic(orc_net* n) {
  if (n->sym_done) return ORC_OK;
  int nb = n->nb;
  int W = (nb + 63) / 64;
  uint64_t* adj = (uint64_t*)xcalloc((size_t)nb * (size_t)W, sizeof(uint64_t));
  uint64_t* pqmask = (uint64_t*)xcalloc((size_t)W, sizeof(uint64_t));
  if (!adj || !pqmask) return ORC_ENOMEM;
#define ADJ(i) (adj + (size_t)(i) * (size_t)W)
  for (int i = 0; i < nb; i++)
    if (n->type[i] == BUS_PQ) pqmask[i >> 6] |= (uint64_t)1 << (i & 63);
  for (int l = 0; l < n->nl; l++) {
    int a = n->f[l], b = n->t[l];
    if (a == n->ref || b == n->ref) continue;
    ADJ(a)[b >> 6] |= (uint64_t)1 << (b & 63);
    ADJ(b)[a >> 6] |= (uint64_t)1 << (a & 63);
  }
  int* alive = (int*)xcalloc((size_t)nb, sizeof(int));
  long* deg = (long*)xcalloc((size_t)nb, sizeof(long));
  int nsb = 0;
  for (int i = 0; i < nb; i++)
    if (n->type[i] != BUS_REF) {
      alive[i] = 1;
      nsb++;
    }
  for (int i = 0; i < nb; i++) {
    if (!alive[i]) continue;
    long d = 0;
    for (int w = 0; w < W; w++)
      d += __builtin_popcountll(ADJ(i)[w]) + __builtin_popcountll(ADJ(i)[w] & pqmask[w]);
    deg[i] = d;
  }
  n->nsb = nsb;
  n->bus_order = (int*)xcalloc((size_t)nsb, sizeof(int));
  /* struct lists: buses adjacent at elimination time (all later in the order) */
  int** st = (int**)xcalloc((size_t)nb, sizeof(int*));
  int* stn = (int*)xcalloc((size_t)nb, sizeof(int));
  int* nbr = (int*)xcalloc((size_t)nb, sizeof(int));
  for (int step = 0; step < nsb; step++) {
    int p = -1;
    for (int i = 0; i < nb; i++)
      if (alive[i] && (p < 0 || deg[i] < deg[p])) p = i; /* ties: smallest id first */
    n->bus_order[step] = p;
    alive[p] = 0;
    int cnt = 0;
    for (int w = 0; w < W; w++) {
      uint64_t bits = ADJ(p)[w];
      while (bits) {
        int b = __builtin_ctzll(bits);
        bits &= bits - 1;
        nbr[cnt++] = w * 64 + b;
      }
    }
    st[p] = (int*)xcalloc((size_t)cnt, sizeof(int));
    memcpy(st[p], nbr, sizeof(int) * (size_t)cnt);
    stn[p] = cnt;
    for (int k = 0; k < cnt; k++) {
      int q = nbr[k];
      uint64_t* aq = ADJ(q);
      for (int w = 0; w < W; w++) aq[w] |= ADJ(p)[w];
      aq[q >> 6] &= ~((uint64_t)1 << (q & 63));
      aq[p >> 6] &= ~((uint64_t)1 << (p & 63));
      long d = 0;
      for (int w = 0; w < W; w++)
        d += __builtin_popcountll(aq[w]) + __builtin_popcountll(aq[w] & pqmask[w]);
      deg[q] = d;
    }
    memset(ADJ(p), 0, sizeof(uint64_t) * (size_t)W);
  }
#undef ADJ
  /* variable order: bus by bus, theta then v */
  int nx = n->nx;
  int* vstart = (int*)xcalloc((size_t)nb, sizeof(int));
  int* wb = (int*)xcalloc((size_t)nb, sizeof(int));
  n->perm = (int*)xcalloc((size_t)nx, sizeof(int));
  n->iperm = (int*)xcalloc((size_t)nx, sizeof(int));
  int k = 0;
  for (int s = 0; s < nsb; s++) {
    int bus = n->bus_order[s];
    vstart[bus] = k;
    n->perm[k++] = n->xth[bus];
    wb[bus] = 1;
    if (n->type[bus] == BUS_PQ) {
      n->perm[k++] = n->xv[bus];
      wb[bus] = 2;
    }
  }
  for (int i = 0; i < nx; i++) n->iperm[n->perm[i]] = i;
  /* lower pattern per row (new indices) from the bus elimination structure */
  int* lcnt = (int*)xcalloc((size_t)nx, sizeof(int));
  for (int s = 0; s < nsb; s++) {
    int bus = n->bus_order[s];
    if (wb[bus] == 2) lcnt[vstart[bus] + 1] += 1;
    for (int q = 0; q < stn[bus]; q++) {
      int ob = st[bus][q];
      for (int r = 0; r < wb[ob]; r++) lcnt[vstart[ob] + r] += wb[bus];
    }
  }
  int** low = (int**)xcalloc((size_t)nx, sizeof(int*));
  int* lfill = (int*)xcalloc((size_t)nx, sizeof(int));
  for (int i = 0; i < nx; i++) low[i] = (int*)xcalloc((size_t)lcnt[i], sizeof(int));
  for (int s = 0; s < nsb; s++) {
    int bus = n->bus_order[s];
    if (wb[bus] == 2) {
      int r = vstart[bus] + 1;
      low[r][lfill[r]++] = vstart[bus];
    }
    for (int q = 0; q < stn[bus]; q++) {
      int ob = st[bus][q];
      for (int r = 0; r < wb[ob]; r++)
        for (int c = 0; c < wb[bus]; c++) low[vstart[ob] + r][lfill[vstart[ob] + r]++] = vstart[bus] + c;
    }
  }
  /* upper pattern = transpose of lower */
  int* ucnt = (int*)xcalloc((size_t)nx, sizeof(int));
  for (int i = 0; i < nx; i++)
    for (int p = 0; p < lcnt[i]; p++) ucnt[low[i][p]]++;
  n->rp = (int*)xcalloc((size_t)nx + 1, sizeof(int));
  for (int i = 0; i < nx; i++) n->rp[i + 1] = n->rp[i] + lcnt[i] + 1 + ucnt[i];
  n->nnz = n->rp[nx];
  n->ci = (int*)xcalloc((size_t)n->nnz, sizeof(int));
  n->dp = (int*)xcalloc((size_t)nx, sizeof(int));
  int* fillp = (int*)xcalloc((size_t)nx, sizeof(int));
  for (int i = 0; i < nx; i++) fillp[i] = n->rp[i];
  for (int i = 0; i < nx; i++)
    for (int p = 0; p < lcnt[i]; p++) n->ci[fillp[i]++] = low[i][p];
  for (int i = 0; i < nx; i++) n->ci[fillp[i]++] = i;
  for (int i = 0; i < nx; i++)
    for (int p = 0; p < lcnt[i]; p++) {
      int j = low[i][p];
      n->ci[fillp[j]++] = i;
    }
  /* sort rows (insertion sort; rows are short) */
  for (int i = 0; i < nx; i++) {
    int b = n->rp[i], e = n->rp[i + 1];
    for (int p = b + 1; p < e; p++) {
      int key = n->ci[p], q = p - 1;
      while (q >= b && n->ci[q] > key) {
        n->ci[q + 1] = n->ci[q];
        q--;
      }
      n->ci[q + 1] = key;
    }
    for (int p = b; p < e; p++)
      if (n->ci[p] == i) n->dp[i] = p;
  }
  /* level sets: forward (lower part) and backward (upper part) */
  n->lev_f = (int*)xcalloc((size_t)nx, sizeof(int));
  n->lev_b = (int*)xcalloc((size_t)nx, sizeof(int));
  for (int i = 0; i < nx; i++) {
    int lv = 0;
    for (int p = n->rp[i]; p < n->dp[i]; p++)
      if (n->lev_f[n->ci[p]] + 1 > lv) lv = n->lev_f[n->ci[p]] + 1;
    n->lev_f[i] = lv;
  }
  for (int i = nx - 1; i >= 0; i--) {
    int lv = 0;
    for (int p = n->dp[i] + 1; p < n->rp[i + 1]; p++)
      if (n->lev_b[n->ci[p]] + 1 > lv) lv = n->lev_b[n->ci[p]] + 1;
    n->lev_b[i] = lv;
  }
  for (int i = 0; i < nx; i++) free(low[i]);
  for (int i = 0; i < nb; i++) free(st[i]);
  free(low);
  free(lfill);
  free(lcnt);
  free(ucnt);
  free(fillp);
  free(st);
  free(stn);
  free(nbr);
  free(vstart);
  free(wb);
  free(alive);
  free(deg);
  free(adj);
  free(pqmask);
  n->sym_done = 1;
  return ORC_OK;
}

int orc_symbolic_sizes(orc_net* n, int* nnz_full, int* n_state_bus) {
  int rc = symbolic(n);
  if (rc) return rc;
  if (nnz_full) *nnz_full = n->nnz;
  if (n_state_bus) *n_state_bus = n->nsb;
  return ORC_OK;
}

int orc_symbolic_export(orc_net* n, int* bus_order, int* perm, int* rowptr, int* colidx,
                        int* lev_f, int* lev_b) {
  int rc = symbolic(n);
  if (rc) return rc;
  if (bus_order) memcpy(bus_order, n->bus_order, sizeof(int) * (size_t)n->nsb);
  if (perm) memcpy(perm, n->perm, sizeof(int) * (size_t)n->nx);
  if (rowptr) memcpy(rowptr, n->rp, sizeof(int) * ((size_t)n->nx + 1));
  if (colidx) memcpy(colidx, n->ci, sizeof(int) * (size_t)n->nnz);
  if (lev_f) memcpy(lev_f, n->lev_f, sizeof(int) * (size_t)n->nx);
  if (lev_b) memcpy(lev_b, n->lev_b, sizeof(int) * (size_t)n->nx);
  return ORC_OK;
}

/* ------------------------------------------------ sparse LU (no pivoting) */

typedef struct {
  int n;
  double* val; /* on the filled pattern: strictly lower = L (unit diag), rest = U */
} lu_t;

/* Factor A = P G_x P^T on the filled pattern, row by row (up-looking). */
static int lu_factor(orc_net* n, const csr_t* Gx, lu_t* lu) {
  int nx = n->nx;
  lu->n = nx;
  lu->val = (double*)xcalloc((size_t)n->nnz, sizeof(double));
  double* w = (double*)xcalloc((size_t)nx, sizeof(double));
  int rc = ORC_OK;
  for (int i = 0; i < nx && rc == ORC_OK; i++) {
    int orow = n->perm[i];
    double rowmax = 0.0;
    for (int p = Gx->rp[orow]; p < Gx->rp[orow + 1]; p++) {
      w[n->iperm[Gx->ci[p]]] += Gx->v[p];
      if (fabs(Gx->v[p]) > rowmax) rowmax = fabs(Gx->v[p]);
    }
    for (int p = n->rp[i]; p < n->dp[i]; p++) {
      int j = n->ci[p];
      double lij = w[j] / lu->val[n->dp[j]];
      lu->val[p] = lij;
      w[j] = 0.0;
      for (int q = n->dp[j] + 1; q < n->rp[j + 1]; q++) w[n->ci[q]] -= lij * lu->val[q];
    }
    for (int p = n->dp[i]; p < n->rp[i + 1]; p++) {
      lu->val[p] = w[n->ci[p]];
      w[n->ci[p]] = 0.0;
    }
    double piv = lu->val[n->dp[i]];
    if (!(fabs(piv) > 1e-14 * rowmax)) rc = ORC_ESINGULAR;
  }
  free(w);
  return rc;
}

/* Solve G_x z = b (transposed = 0) or G_x^T z = b (transposed = 1). */
static void lu_solve(const orc_net* n, const lu_t* lu, const double* b, double* z, int transposed) {
  int nx = n->nx;
  double* y = (double*)xcalloc((size_t)nx, sizeof(double));
  for (int i = 0; i < nx; i++) y[i] = b[n->perm[i]];
  if (!transposed) {
    for (int i = 0; i < nx; i++) { /* L y = b */
      double s = y[i];
      for (int p = n->rp[i]; p < n->dp[i]; p++) s -= lu->val[p] * y[n->ci[p]];
      y[i] = s;
    }
    for (int i = nx - 1; i >= 0; i--) { /* U z = y */
      double s = y[i];
      for (int p = n->dp[i] + 1; p < n->rp[i + 1]; p++) s -= lu->val[p] * y[n->ci[p]];
      y[i] = s / lu->val[n->dp[i]];
    }
  } else {
    for (int j = 0; j < nx; j++) { /* U^T y = b, column-oriented on the rows of U */
      y[j] /= lu->val[n->dp[j]];
      for (int p = n->dp[j] + 1; p < n->rp[j + 1]; p++) y[n->ci[p]] -= lu->val[p] * y[j];
    }
    for (int j = nx - 1; j >= 0; j--) { /* L^T z = y */
      for (int p = n->rp[j]; p < n->dp[j]; p++) y[n->ci[p]] -= lu->val[p] * y[j];
    }
  }
  for (int i = 0; i < nx; i++) z[n->perm[i]] = y[i];
  free(y);
}

/* ------------------------------------------------------- branch flows */

/* One end of a branch: flows out of bus s towards bus o and their first and
 * second derivatives w.r.t. the local variables (v_s, v_o, theta_s, theta_o). */
typedef struct {
  double P, Q;
  double dP[4], dQ[4];
  double hP[4][4], hQ[4][4];
} side_t;

static void side_flow(double vs, double vo, double ang, double Gss, double Bss, double Gso,
                      double Bso, side_t* o) {
  double cs = cos(ang), sn = sin(ang);
  double A = Gso * cs + Bso * sn;  /* d/dang A = -Bq */
  double Bq = Gso * sn - Bso * cs; /* d/dang Bq = A  */
  o->P = vs * vs * Gss + vs * vo * A;
  o->Q = -vs * vs * Bss + vs * vo * Bq;
  o->dP[0] = 2.0 * vs * Gss + vo * A;
  o->dP[1] = vs * A;
  o->dP[2] = -vs * vo * Bq;
  o->dP[3] = vs * vo * Bq;
  o->dQ[0] = -2.0 * vs * Bss + vo * Bq;
  o->dQ[1] = vs * Bq;
  o->dQ[2] = vs * vo * A;
  o->dQ[3] = -vs * vo * A;
  double hp[4][4] = {{2.0 * Gss, A, -vo * Bq, vo * Bq},
                     {A, 0.0, -vs * Bq, vs * Bq},
                     {-vo * Bq, -vs * Bq, -vs * vo * A, vs * vo * A},
                     {vo * Bq, vs * Bq, vs * vo * A, -vs * vo * A}};
  double hq[4][4] = {{-2.0 * Bss, Bq, vo * A, -vo * A},
                     {Bq, 0.0, vs * A, -vs * A},
                     {vo * A, vs * A, -vs * vo * Bq, vs * vo * Bq},
                     {-vo * A, -vs * A, vs * vo * Bq, -vs * vo * Bq}};
  memcpy(o->hP, hp, sizeof(hp));
  memcpy(o->hQ, hq, sizeof(hq));
}

/* bus voltages from (x, u) */
static void unpack(const orc_net* n, const double* x, const double* u, double* v, double* th) {
  for (int i = 0; i < n->nb; i++) {
    v[i] = (n->type[i] == BUS_PQ) ? x[n->xv[i]] : u[n->zv[i] - n->nx];
    th[i] = (n->type[i] == BUS_REF) ? 0.0 : x[n->xth[i]];
  }
}

static void branch_sides(const orc_net* n, const double* v, const double* th, int l, side_t* sf,
                         side_t* stt) {
  int a = n->f[l], b = n->t[l];
  side_flow(v[a], v[b], th[a] - th[b], n->Gff[l], n->Bff[l], n->Gft[l], n->Bft[l], sf);
  side_flow(v[b], v[a], th[b] - th[a], n->Gtt[l], n->Btt[l], n->Gtf[l], n->Btf[l], stt);
}

/* z indices of the local variables (v_s, v_o, theta_s, theta_o) */
static void local_z(const orc_net* n, int s, int o, int zi[4]) {
  zi[0] = n->zv[s];
  zi[1] = n->zv[o];
  zi[2] = n->zth[s];
  zi[3] = n->zth[o];
}

int orc_eval(orc_net* n, const double* x, const double* u, const double* pd, const double* qd,
             double* g, double* c, double* P, double* Q, double* f_cost) {
  int nb = n->nb, nl = n->nl;
  double* v = (double*)xcalloc((size_t)nb, sizeof(double));
  double* th = (double*)xcalloc((size_t)nb, sizeof(double));
  double* Pi = (double*)xcalloc((size_t)nb, sizeof(double));
  double* Qi = (double*)xcalloc((size_t)nb, sizeof(double));
  unpack(n, x, u, v, th);
  for (int l = 0; l < nl; l++) {
    side_t sf, st;
    branch_sides(n, v, th, l, &sf, &st);
    Pi[n->f[l]] += sf.P;
    Qi[n->f[l]] += sf.Q;
    Pi[n->t[l]] += st.P;
    Qi[n->t[l]] += st.Q;
    if (c) {
      c[l] = sf.P * sf.P + sf.Q * sf.Q;
      c[nl + l] = st.P * st.P + st.Q * st.Q;
    }
  }
  if (g) {
    for (int i = 0; i < nb; i++) {
      if (n->type[i] == BUS_REF) continue;
      double pg = (n->type[i] == BUS_PV) ? u[1 + n->npv + n->pvpos[i]] : 0.0;
      g[n->xth[i]] = Pi[i] - pg + pd[i];
      if (n->type[i] == BUS_PQ) g[n->xv[i]] = Qi[i] + qd[i];
    }
  }
  if (c) {
    int o = 2 * nl;
    for (int k = 0; k < n->npq; k++) c[o + k] = v[n->pq[k]];
    o += n->npq;
    c[o] = Pi[n->ref] + pd[n->ref];
    c[o + 1] = Qi[n->ref] + qd[n->ref];
    o += 2;
    for (int k = 0; k < n->npv; k++) c[o + k] = Qi[n->pv[k]] + qd[n->pv[k]];
  }
  if (f_cost) {
    double fc = 0.0;
    for (int gI = 0; gI < n->ng; gI++) {
      int bus = n->gbus[gI];
      double p = (bus == n->ref) ? Pi[bus] + pd[bus] : u[1 + n->npv + n->pvpos[bus]];
      fc += n->c2[gI] * p * p + n->c1[gI] * p + n->c0[gI];
    }
    *f_cost = fc;
  }
  if (P) memcpy(P, Pi, sizeof(double) * (size_t)nb);
  if (Q) memcpy(Q, Qi, sizeof(double) * (size_t)nb);
  free(v);
  free(th);
  free(Pi);
  free(Qi);
  return ORC_OK;
}

/* Jacobian of g w.r.t. z = (x, u): n_x rows, n_x + n_u columns. */
static csr_t jac_g(const orc_net* n, const double* v, const double* th) {
  coo_t a = {0};
  for (int l = 0; l < n->nl; l++) {
    side_t sd[2];
    branch_sides(n, v, th, l, &sd[0], &sd[1]);
    for (int e = 0; e < 2; e++) {
      int s = e ? n->t[l] : n->f[l], o = e ? n->f[l] : n->t[l];
      int zi[4];
      local_z(n, s, o, zi);
      if (n->type[s] == BUS_REF) continue;
      for (int k = 0; k < 4; k++) {
        coo_add(&a, n->xth[s], zi[k], sd[e].dP[k]);
        if (n->type[s] == BUS_PQ) coo_add(&a, n->xv[s], zi[k], sd[e].dQ[k]);
      }
    }
  }
  for (int k = 0; k < n->npv; k++) coo_add(&a, n->xth[n->pv[k]], n->nx + 1 + n->npv + k, -1.0);
  csr_t J = coo_to_csr(&a, n->nx, n->nx + n->nu);
  coo_free(&a);
  return J;
}

/* Jacobian of c w.r.t. z: m rows. */
static csr_t jac_c(const orc_net* n, const double* v, const double* th) {
  coo_t a = {0};
  int nl = n->nl;
  int o_v = 2 * nl, o_r = 2 * nl + n->npq;
  for (int l = 0; l < nl; l++) {
    side_t sd[2];
    branch_sides(n, v, th, l, &sd[0], &sd[1]);
    for (int e = 0; e < 2; e++) {
      int s = e ? n->t[l] : n->f[l], o = e ? n->f[l] : n->t[l];
      int zi[4];
      local_z(n, s, o, zi);
      for (int k = 0; k < 4; k++) {
        coo_add(&a, e * nl + l, zi[k], 2.0 * (sd[e].P * sd[e].dP[k] + sd[e].Q * sd[e].dQ[k]));
        if (s == n->ref) {
          coo_add(&a, o_r, zi[k], sd[e].dP[k]);
          coo_add(&a, o_r + 1, zi[k], sd[e].dQ[k]);
        } else if (n->type[s] == BUS_PV) {
          coo_add(&a, o_r + 2 + n->pvpos[s], zi[k], sd[e].dQ[k]);
        }
      }
    }
  }
  for (int k = 0; k < n->npq; k++) coo_add(&a, o_v + k, n->zv[n->pq[k]], 1.0);
  csr_t J = coo_to_csr(&a, n->m, n->nx + n->nu);
  coo_free(&a);
  return J;
}

/* first-order AL weights phi'_i = y_i sigma_i + rho sigma_i^2 (c_i - s_i) and F */
static double al_weights(const orc_net* n, const double* c, double fcost, double sigma_f, double rho,
                         const double* sigma_c, const double* y, const double* s, double* phid) {
  double F = sigma_f * fcost;
  for (int i = 0; i < n->m; i++) {
    double r = c[i] - s[i];
    F += y[i] * sigma_c[i] * r + 0.5 * rho * sigma_c[i] * sigma_c[i] * r * r;
    phid[i] = y[i] * sigma_c[i] + rho * sigma_c[i] * sigma_c[i] * r;
  }
  return F;
}

/* gradient of F w.r.t. z (partial derivatives, x and u together) */
static void grad_F_z(const orc_net* n, const csr_t* Jc, const double* P, const double* u,
                     const double* pd, double sigma_f, const double* phid, double* dF) {
  csr_mtv(Jc, phid, dF);
  /* objective: slack generator through p_ref = P_ref + pd_ref; PV through p_pv */
  int gr = n->gen_at[n->ref];
  double pref = P[n->ref] + pd[n->ref];
  double wref = sigma_f * (2.0 * n->c2[gr] * pref + n->c1[gr]);
  /* row o_r of Jc is grad P_ref: add wref times it */
  int o_r = 2 * n->nl + n->npq;
  for (int p = Jc->rp[o_r]; p < Jc->rp[o_r + 1]; p++) dF[Jc->ci[p]] += wref * Jc->v[p];
  for (int k = 0; k < n->npv; k++) {
    int gI = n->gen_at[n->pv[k]];
    double pk = u[1 + n->npv + k];
    dF[n->nx + 1 + n->npv + k] += sigma_f * (2.0 * n->c2[gI] * pk + n->c1[gI]);
  }
}

/* split a CSR over z columns into G_x (columns < nx) */
static csr_t take_x(const orc_net* n, const csr_t* J) {
  coo_t a = {0};
  for (int i = 0; i < J->nr; i++)
    for (int p = J->rp[i]; p < J->rp[i + 1]; p++)
      if (J->ci[p] < n->nx) coo_add(&a, i, J->ci[p], J->v[p]);
  csr_t r = coo_to_csr(&a, J->nr, n->nx);
  coo_free(&a);
  return r;
}

/* ----------------------------------------------------------- power flow */

int orc_powerflow(orc_net* n, const double* u, const double* pd, const double* qd,
                  double* x_inout, double tol, int max_it, int* iters, double* res2,
                  double* resinf) {
  int rc = symbolic(n);
  if (rc) return rc;
  int nx = n->nx, nb = n->nb;
  double* g = (double*)xcalloc((size_t)nx, sizeof(double));
  double* d = (double*)xcalloc((size_t)nx, sizeof(double));
  double* v = (double*)xcalloc((size_t)nb, sizeof(double));
  double* th = (double*)xcalloc((size_t)nb, sizeof(double));
  int it = 0;
  rc = ORC_ENOCONV;
  double nrm2 = 0.0, nrmi = 0.0;
  for (it = 0;; it++) {
    orc_eval(n, x_inout, u, pd, qd, g, NULL, NULL, NULL, NULL);
    nrm2 = 0.0;
    nrmi = 0.0;
    for (int i = 0; i < nx; i++) {
      nrm2 += g[i] * g[i];
      if (fabs(g[i]) > nrmi) nrmi = fabs(g[i]);
    }
    nrm2 = sqrt(nrm2);
    if (!isfinite(nrm2)) {
      rc = ORC_ENOCONV;
      break;
    }
    if (nrm2 < tol) {
      rc = ORC_OK;
      break;
    }
    if (it >= max_it) break;
    unpack(n, x_inout, u, v, th);
    csr_t J = jac_g(n, v, th);
    csr_t Gx = take_x(n, &J);
    lu_t lu;
    int frc = lu_factor(n, &Gx, &lu);
    if (frc == ORC_OK) lu_solve(n, &lu, g, d, 0);
    free(lu.val);
    csr_free(&J);
    csr_free(&Gx);
    if (frc) {
      rc = frc;
      break;
    }
    for (int i = 0; i < nx; i++) x_inout[i] -= d[i];
  }
  if (iters) *iters = it;
  if (res2) *res2 = nrm2;
  if (resinf) *resinf = nrmi;
  free(g);
  free(d);
  free(v);
  free(th);
  return rc;
}

/* ------------------------------------------------------- reduced gradient */

typedef struct {
  double *v, *th, *P, *Q, *c, *phid, *dF, *lam;
  double F, fcost;
  csr_t Jg, Jc, Gx;
  lu_t lu;
} state_t;

static void state_free(state_t* S) {
  free(S->v);
  free(S->th);
  free(S->P);
  free(S->Q);
  free(S->c);
  free(S->phid);
  free(S->dF);
  free(S->lam);
  csr_free(&S->Jg);
  csr_free(&S->Jc);
  csr_free(&S->Gx);
  free(S->lu.val);
}

/* evaluate everything the gradient and the Hessian need at (x, u) */
static int state_build(orc_net* n, const double* x, const double* u, const double* pd,
                       const double* qd, double sigma_f, double rho, const double* sigma_c,
                       const double* y, const double* s, state_t* S) {
  memset(S, 0, sizeof(*S));
  int rc = symbolic(n);
  if (rc) return rc;
  int nb = n->nb, nx = n->nx, nz = n->nx + n->nu, m = n->m;
  S->v = (double*)xcalloc((size_t)nb, sizeof(double));
  S->th = (double*)xcalloc((size_t)nb, sizeof(double));
  S->P = (double*)xcalloc((size_t)nb, sizeof(double));
  S->Q = (double*)xcalloc((size_t)nb, sizeof(double));
  S->c = (double*)xcalloc((size_t)m, sizeof(double));
  S->phid = (double*)xcalloc((size_t)m, sizeof(double));
  S->dF = (double*)xcalloc((size_t)nz, sizeof(double));
  S->lam = (double*)xcalloc((size_t)nx, sizeof(double));
  unpack(n, x, u, S->v, S->th);
  orc_eval(n, x, u, pd, qd, NULL, S->c, S->P, S->Q, &S->fcost);
  S->F = al_weights(n, S->c, S->fcost, sigma_f, rho, sigma_c, y, s, S->phid);
  S->Jg = jac_g(n, S->v, S->th);
  S->Jc = jac_c(n, S->v, S->th);
  S->Gx = take_x(n, &S->Jg);
  grad_F_z(n, &S->Jc, S->P, u, pd, sigma_f, S->phid, S->dF);
  rc = lu_factor(n, &S->Gx, &S->lu);
  if (rc) return rc;
  /* first-order adjoint: G_x^T lam = -(d_x F)^T */
  double* rhs = (double*)xcalloc((size_t)nx, sizeof(double));
  for (int i = 0; i < nx; i++) rhs[i] = -S->dF[i];
  lu_solve(n, &S->lu, rhs, S->lam, 1);
  free(rhs);
  return ORC_OK;
}

/* G_u^T psi added into out (n_u) */
static void gu_t_times(const orc_net* n, const csr_t* Jg, const double* psi, double* out) {
  for (int i = 0; i < Jg->nr; i++)
    for (int p = Jg->rp[i]; p < Jg->rp[i + 1]; p++)
      if (Jg->ci[p] >= n->nx) out[Jg->ci[p] - n->nx] += Jg->v[p] * psi[i];
}

/* G_u w into out (n_x) */
static void gu_times(const orc_net* n, const csr_t* Jg, const double* w, double* out) {
  for (int i = 0; i < Jg->nr; i++) {
    double s = 0.0;
    for (int p = Jg->rp[i]; p < Jg->rp[i + 1]; p++)
      if (Jg->ci[p] >= n->nx) s += Jg->v[p] * w[Jg->ci[p] - n->nx];
    out[i] = s;
  }
}

int orc_reduced_gradient(orc_net* n, const double* x, const double* u, const double* pd,
                         const double* qd, double sigma_f, double rho, const double* sigma_c,
                         const double* y, const double* s, double* F, double* grad_u,
                         double* grad_s, double* c, double* lambda, double* grad_pd,
                         double* grad_qd) {
  state_t S;
  int rc = state_build(n, x, u, pd, qd, sigma_f, rho, sigma_c, y, s, &S);
  if (rc) {
    state_free(&S);
    return rc;
  }
  int nx = n->nx, nu = n->nu, m = n->m;
  if (F) *F = S.F;
  if (grad_u) {
    for (int j = 0; j < nu; j++) grad_u[j] = S.dF[nx + j];
    gu_t_times(n, &S.Jg, S.lam, grad_u);
  }
  if (grad_s)
    for (int i = 0; i < m; i++) grad_s[i] = -S.phid[i];
  if (c) memcpy(c, S.c, sizeof(double) * (size_t)m);
  if (lambda) memcpy(lambda, S.lam, sizeof(double) * (size_t)nx);
  int o_r = 2 * n->nl + n->npq;
  int gr = n->gen_at[n->ref];
  double pref = S.P[n->ref] + pd[n->ref];
  if (grad_pd) {
    for (int i = 0; i < n->nb; i++)
      grad_pd[i] = (n->type[i] == BUS_REF)
                       ? sigma_f * (2.0 * n->c2[gr] * pref + n->c1[gr]) + S.phid[o_r]
                       : S.lam[n->xth[i]];
  }
  if (grad_qd) {
    for (int i = 0; i < n->nb; i++) {
      if (n->type[i] == BUS_REF)
        grad_qd[i] = S.phid[o_r + 1];
      else if (n->type[i] == BUS_PV)
        grad_qd[i] = S.phid[o_r + 2 + n->pvpos[i]];
      else
        grad_qd[i] = S.lam[n->xv[i]];
    }
  }
  state_free(&S);
  return ORC_OK;
}

/* -------------------------------------------------------- reduced Hessian */

/* Explicit second derivatives of l = F + lam^T g over z, with GN weights omega. */
static csr_t hess_l(const orc_net* n, const state_t* S, const double* u, const double* pd,
                    double sigma_f, double rho, const double* sigma_c, const double* omega) {
  int nl = n->nl, nb = n->nb, m = n->m;
  int o_v = 2 * nl, o_r = 2 * nl + n->npq;
  double* om = (double*)xcalloc((size_t)m, sizeof(double));
  for (int i = 0; i < m; i++) om[i] = omega ? omega[i] : rho * sigma_c[i] * sigma_c[i];
  int gr = n->gen_at[n->ref];
  double pref = S->P[n->ref] + pd[n->ref];
  /* first-order weights on the injections of each bus */
  double* wP = (double*)xcalloc((size_t)nb, sizeof(double));
  double* wQ = (double*)xcalloc((size_t)nb, sizeof(double));
  for (int i = 0; i < nb; i++) {
    if (n->type[i] == BUS_REF) {
      wP[i] = S->phid[o_r] + sigma_f * (2.0 * n->c2[gr] * pref + n->c1[gr]);
      wQ[i] = S->phid[o_r + 1];
    } else if (n->type[i] == BUS_PV) {
      wP[i] = S->lam[n->xth[i]];
      wQ[i] = S->phid[o_r + 2 + n->pvpos[i]];
    } else {
      wP[i] = S->lam[n->xth[i]];
      wQ[i] = S->lam[n->xv[i]];
    }
  }
  (void)u;
  coo_t a = {0};
  for (int l = 0; l < nl; l++) {
    side_t sd[2];
    branch_sides(n, S->v, S->th, l, &sd[0], &sd[1]);
    for (int e = 0; e < 2; e++) {
      int s = e ? n->t[l] : n->f[l], o = e ? n->f[l] : n->t[l];
      int zi[4];
      local_z(n, s, o, zi);
      const side_t* q = &sd[e];
      double ph = S->phid[e * nl + l], omh = om[e * nl + l];
      double aP = wP[s] + 2.0 * ph * q->P, aQ = wQ[s] + 2.0 * ph * q->Q;
      double gh[4];
      for (int k = 0; k < 4; k++) gh[k] = 2.0 * (q->P * q->dP[k] + q->Q * q->dQ[k]);
      for (int r = 0; r < 4; r++)
        for (int k = 0; k < 4; k++) {
          double val = aP * q->hP[r][k] + aQ * q->hQ[r][k] +
                       2.0 * ph * (q->dP[r] * q->dP[k] + q->dQ[r] * q->dQ[k]) + omh * gh[r] * gh[k];
          coo_add(&a, zi[r], zi[k], val);
        }
    }
  }
  /* bus-level Gauss-Newton terms: omega (grad r)(grad r)^T for p_ref, q_ref, q_pv;
   * plus the curvature 2 sigma_f c2 of the slack cost along grad P_ref */
  for (int rrow = o_r; rrow < m; rrow++) {
    double kap = om[rrow];
    if (rrow == o_r) kap += 2.0 * sigma_f * n->c2[gr];
    for (int p = S->Jc.rp[rrow]; p < S->Jc.rp[rrow + 1]; p++)
      for (int q2 = S->Jc.rp[rrow]; q2 < S->Jc.rp[rrow + 1]; q2++)
        coo_add(&a, S->Jc.ci[p], S->Jc.ci[q2], kap * S->Jc.v[p] * S->Jc.v[q2]);
  }
  for (int k = 0; k < n->npq; k++) coo_add(&a, n->zv[n->pq[k]], n->zv[n->pq[k]], om[o_v + k]);
  for (int k = 0; k < n->npv; k++) {
    int gI = n->gen_at[n->pv[k]];
    int zp = n->nx + 1 + n->npv + k;
    coo_add(&a, zp, zp, 2.0 * sigma_f * n->c2[gI]);
  }
  csr_t K = coo_to_csr(&a, n->nx + n->nu, n->nx + n->nu);
  coo_free(&a);
  free(om);
  free(wP);
  free(wQ);
  return K;
}

/* One adjoint-adjoint HVP (Prop. 2) with prebuilt state and l-Hessian K. */
static void hvp_one(const orc_net* n, const state_t* S, const csr_t* K, const double* w,
                    double* Hw, double* work /* 4 nx + 2 nz */) {
  int nx = n->nx, nu = n->nu, nz = nx + nu;
  double* b = work;
  double* z = b + nx;
  double* rr = z + nx;
  double* psi = rr + nx;
  double* d = psi + nx;
  double* yk = d + nz;
  gu_times(n, &S->Jg, w, b); /* G_x z = -G_u w */
  for (int i = 0; i < nx; i++) b[i] = -b[i];
  lu_solve(n, &S->lu, b, z, 0);
  for (int i = 0; i < nx; i++) d[i] = z[i];
  for (int j = 0; j < nu; j++) d[nx + j] = w[j];
  csr_mv(K, d, yk); /* (l_xx z + l_xu w ; l_ux z + l_uu w) */
  for (int i = 0; i < nx; i++) rr[i] = -yk[i];
  lu_solve(n, &S->lu, rr, psi, 1); /* G_x^T psi = -(l_xu w + l_xx z) */
  for (int j = 0; j < nu; j++) Hw[j] = yk[nx + j];
  gu_t_times(n, &S->Jg, psi, Hw); /* + G_u^T psi */
}

int orc_reduced_hessian(orc_net* n, const double* x, const double* u, const double* pd,
                        const double* qd, double sigma_f, double rho, const double* sigma_c,
                        const double* y, const double* s, const double* omega, const int* cols,
                        int ncols, double* H) {
  state_t S;
  int rc = state_build(n, x, u, pd, qd, sigma_f, rho, sigma_c, y, s, &S);
  if (rc) {
    state_free(&S);
    return rc;
  }
  int nx = n->nx, nu = n->nu;
  for (int c = 0; c < ncols; c++) {
    int j = cols ? cols[c] : c;
    if (j < 0 || j >= nu) rc = ORC_EINVAL;
  }
  if (rc) {
    state_free(&S);
    return rc;
  }
  csr_t K = hess_l(n, &S, u, pd, sigma_f, rho, sigma_c, omega);
  /* The columns are independent HVPs with the same factors (Sec. III-C); with
   * OpenMP (OMP_NUM_THREADS) they are shared out over threads, each with its own
   * work vectors; the arithmetic of a column does not depend on the thread. */
#pragma omp parallel
  {
    double* work = (double*)xcalloc((size_t)(4 * nx + 2 * (nx + nu)), sizeof(double));
    double* w = (double*)xcalloc((size_t)nu, sizeof(double));
#pragma omp for schedule(dynamic, 4)
    for (int c = 0; c < ncols; c++) {
      int j = cols ? cols[c] : c;
      memset(w, 0, sizeof(double) * (size_t)nu);
      w[j] = 1.0;
      hvp_one(n, &S, &K, w, H + (size_t)c * (size_t)nu, work);
    }
    free(work);
    free(w);
  }
  csr_free(&K);
  state_free(&S);
  return rc;
}

int orc_hvp(orc_net* n, const double* x, const double* u, const double* pd, const double* qd,
            double sigma_f, double rho, const double* sigma_c, const double* y, const double* s,
            const double* omega, const double* w, double* Hw) {
  state_t S;
  int rc = state_build(n, x, u, pd, qd, sigma_f, rho, sigma_c, y, s, &S);
  if (rc) {
    state_free(&S);
    return rc;
  }
  int nx = n->nx, nu = n->nu;
  csr_t K = hess_l(n, &S, u, pd, sigma_f, rho, sigma_c, omega);
  double* work = (double*)xcalloc((size_t)(4 * nx + 2 * (nx + nu)), sizeof(double));
  hvp_one(n, &S, &K, w, Hw, work);
  free(work);
  csr_free(&K);
  state_free(&S);
  return ORC_OK;
}

int orc_reduced_jac_prod(orc_net* n, const double* x, const double* u, const double* pd,
                         const double* qd, const double* v, double* Jv, const double* w,
                         double* Jtw) {
  int rc = symbolic(n);
  if (rc) return rc;
  int nb = n->nb, nx = n->nx, nu = n->nu, m = n->m, nz = nx + nu;
  double* vb = (double*)xcalloc((size_t)nb, sizeof(double));
  double* th = (double*)xcalloc((size_t)nb, sizeof(double));
  unpack(n, x, u, vb, th);
  csr_t Jg = jac_g(n, vb, th);
  csr_t Jc = jac_c(n, vb, th);
  csr_t Gx = take_x(n, &Jg);
  lu_t lu;
  rc = lu_factor(n, &Gx, &lu);
  double* tmp = (double*)xcalloc((size_t)nz, sizeof(double));
  double* z = (double*)xcalloc((size_t)nz, sizeof(double));
  if (rc == ORC_OK && v && Jv) { /* J v = d_u c v + d_x c z, G_x z = -G_u v */
    gu_times(n, &Jg, v, tmp);
    for (int i = 0; i < nx; i++) tmp[i] = -tmp[i];
    lu_solve(n, &lu, tmp, z, 0);
    for (int j = 0; j < nu; j++) z[nx + j] = v[j];
    csr_mv(&Jc, z, Jv);
  }
  if (rc == ORC_OK && w && Jtw) { /* J^T w = d_u c^T w + G_u^T mu, G_x^T mu = -d_x c^T w */
    double* ctw = (double*)xcalloc((size_t)nz, sizeof(double));
    csr_mtv(&Jc, w, ctw);
    for (int i = 0; i < nx; i++) tmp[i] = -ctw[i];
    lu_solve(n, &lu, tmp, z, 1);
    for (int j = 0; j < nu; j++) Jtw[j] = ctw[nx + j];
    gu_t_times(n, &Jg, z, Jtw);
    free(ctw);
  }
  (void)m;
  free(tmp);
  free(z);
  free(lu.val);
  csr_free(&Jg);
  csr_free(&Jc);
  csr_free(&Gx);
  free(vb);
  free(th);
  return rc;
}

/* ------------------------------------------------ brute force (hyper-dual) */

/* hyper-dual number a + b e1 + c e2 + d e1 e2, with e1^2 = e2^2 = 0 */
typedef struct {
  double a, b, c, d;
} hd;

static hd hd_c(double a) { hd r = {a, 0, 0, 0}; return r; }
static hd hd_add(hd x, hd y) { hd r = {x.a + y.a, x.b + y.b, x.c + y.c, x.d + y.d}; return r; }
static hd hd_sub(hd x, hd y) { hd r = {x.a - y.a, x.b - y.b, x.c - y.c, x.d - y.d}; return r; }
static hd hd_mul(hd x, hd y) {
  hd r = {x.a * y.a, x.a * y.b + x.b * y.a, x.a * y.c + x.c * y.a,
          x.a * y.d + x.b * y.c + x.c * y.b + x.d * y.a};
  return r;
}
static hd hd_scale(hd x, double s) { hd r = {s * x.a, s * x.b, s * x.c, s * x.d}; return r; }
/* f(x) for smooth f with f', f'' at x.a: f(a) + f'(a)(b e1 + c e2 + d e1e2) + f''(a) b c e1e2 */
static hd hd_fun(hd x, double f0, double f1, double f2) {
  hd r = {f0, f1 * x.b, f1 * x.c, f1 * x.d + f2 * x.b * x.c};
  return r;
}
static hd hd_cos(hd x) { return hd_fun(x, cos(x.a), -sin(x.a), -cos(x.a)); }
static hd hd_sin(hd x) { return hd_fun(x, sin(x.a), cos(x.a), -sin(x.a)); }

typedef struct {
  hd re, im;
} chd;

static chd chd_mulc(double yr, double yi, chd v) { /* (yr + j yi) v */
  chd r = {hd_sub(hd_scale(v.re, yr), hd_scale(v.im, yi)),
           hd_add(hd_scale(v.im, yr), hd_scale(v.re, yi))};
  return r;
}

/* S = V conj(I): returns P + jQ */
static chd chd_power(chd V, chd I) {
  chd r = {hd_add(hd_mul(V.re, I.re), hd_mul(V.im, I.im)),
           hd_sub(hd_mul(V.im, I.re), hd_mul(V.re, I.im))};
  return r;
}

typedef struct {
  const orc_net* n;
  double *Yr, *Yi; /* dense bus admittance */
  double *Yffr, *Yffi, *Yftr, *Yfti, *Ytfr, *Ytfi, *Yttr, *Ytti;
  const double *pd, *qd;
} bf_t;

/* evaluate g (nx), c (m), cost with hyper-dual inputs z (nx + nu) */
static void bf_eval(const bf_t* B, const hd* z, hd* g, hd* c, hd* cost) {
  const orc_net* n = B->n;
  int nb = n->nb, nl = n->nl, nx = n->nx;
  chd* V = (chd*)xcalloc((size_t)nb, sizeof(chd));
  chd* S = (chd*)xcalloc((size_t)nb, sizeof(chd));
  for (int i = 0; i < nb; i++) {
    hd vm = (n->type[i] == BUS_PQ) ? z[n->xv[i]] : z[n->zv[i]];
    hd ang = (n->type[i] == BUS_REF) ? hd_c(0.0) : z[n->xth[i]];
    V[i].re = hd_mul(vm, hd_cos(ang));
    V[i].im = hd_mul(vm, hd_sin(ang));
  }
  for (int i = 0; i < nb; i++) {
    chd I = {hd_c(0.0), hd_c(0.0)};
    for (int k = 0; k < nb; k++) {
      double yr = B->Yr[(size_t)i * nb + k], yi = B->Yi[(size_t)i * nb + k];
      if (yr == 0.0 && yi == 0.0) continue;
      chd t = chd_mulc(yr, yi, V[k]);
      I.re = hd_add(I.re, t.re);
      I.im = hd_add(I.im, t.im);
    }
    S[i] = chd_power(V[i], I);
  }
  if (c) {
    for (int l = 0; l < nl; l++) {
      int a = n->f[l], b = n->t[l];
      chd If = chd_mulc(B->Yffr[l], B->Yffi[l], V[a]);
      chd t1 = chd_mulc(B->Yftr[l], B->Yfti[l], V[b]);
      If.re = hd_add(If.re, t1.re);
      If.im = hd_add(If.im, t1.im);
      chd It = chd_mulc(B->Yttr[l], B->Ytti[l], V[b]);
      chd t2 = chd_mulc(B->Ytfr[l], B->Ytfi[l], V[a]);
      It.re = hd_add(It.re, t2.re);
      It.im = hd_add(It.im, t2.im);
      chd Sf = chd_power(V[a], If), St = chd_power(V[b], It);
      c[l] = hd_add(hd_mul(Sf.re, Sf.re), hd_mul(Sf.im, Sf.im));
      c[nl + l] = hd_add(hd_mul(St.re, St.re), hd_mul(St.im, St.im));
    }
    int o = 2 * nl;
    for (int k = 0; k < n->npq; k++) c[o + k] = z[n->xv[n->pq[k]]];
    o += n->npq;
    c[o] = hd_add(S[n->ref].re, hd_c(B->pd[n->ref]));
    c[o + 1] = hd_add(S[n->ref].im, hd_c(B->qd[n->ref]));
    o += 2;
    for (int k = 0; k < n->npv; k++) c[o + k] = hd_add(S[n->pv[k]].im, hd_c(B->qd[n->pv[k]]));
  }
  if (g) {
    for (int i = 0; i < nb; i++) {
      if (n->type[i] == BUS_REF) continue;
      hd pg = (n->type[i] == BUS_PV) ? z[nx + 1 + n->npv + n->pvpos[i]] : hd_c(0.0);
      g[n->xth[i]] = hd_add(hd_sub(S[i].re, pg), hd_c(B->pd[i]));
      if (n->type[i] == BUS_PQ) g[n->xv[i]] = hd_add(S[i].im, hd_c(B->qd[i]));
    }
  }
  if (cost) {
    hd fc = hd_c(0.0);
    for (int gI = 0; gI < n->ng; gI++) {
      int bus = n->gbus[gI];
      hd p = (bus == n->ref) ? hd_add(S[bus].re, hd_c(B->pd[bus]))
                             : z[nx + 1 + n->npv + n->pvpos[bus]];
      fc = hd_add(fc, hd_add(hd_scale(hd_mul(p, p), n->c2[gI]),
                             hd_add(hd_scale(p, n->c1[gI]), hd_c(n->c0[gI]))));
    }
    *cost = fc;
  }
  free(V);
  free(S);
}

/* dense LU with partial pivoting; A is n x n row-major, overwritten */
static int dense_lu(int n, double* A, int* piv) {
  for (int k = 0; k < n; k++) {
    int p = k;
    for (int i = k + 1; i < n; i++)
      if (fabs(A[(size_t)i * n + k]) > fabs(A[(size_t)p * n + k])) p = i;
    piv[k] = p;
    if (A[(size_t)p * n + k] == 0.0) return ORC_ESINGULAR;
    if (p != k)
      for (int j = 0; j < n; j++) {
        double t = A[(size_t)k * n + j];
        A[(size_t)k * n + j] = A[(size_t)p * n + j];
        A[(size_t)p * n + j] = t;
      }
    for (int i = k + 1; i < n; i++) {
      double l = A[(size_t)i * n + k] / A[(size_t)k * n + k];
      A[(size_t)i * n + k] = l;
      for (int j = k + 1; j < n; j++) A[(size_t)i * n + j] -= l * A[(size_t)k * n + j];
    }
  }
  return ORC_OK;
}

/* solve with the factors of dense_lu: A x = b (trans = 0) or A^T x = b (trans = 1) */
static void dense_lu_solve(int n, const double* A, const int* piv, double* b, int trans) {
  if (!trans) {
    for (int k = 0; k < n; k++) {
      double t = b[k];
      b[k] = b[piv[k]];
      b[piv[k]] = t;
    }
    for (int i = 0; i < n; i++)
      for (int j = 0; j < i; j++) b[i] -= A[(size_t)i * n + j] * b[j];
    for (int i = n - 1; i >= 0; i--) {
      for (int j = i + 1; j < n; j++) b[i] -= A[(size_t)i * n + j] * b[j];
      b[i] /= A[(size_t)i * n + i];
    }
  } else {
    for (int i = 0; i < n; i++) {
      for (int j = 0; j < i; j++) b[i] -= A[(size_t)j * n + i] * b[j];
      b[i] /= A[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; i--)
      for (int j = i + 1; j < n; j++) b[i] -= A[(size_t)j * n + i] * b[j];
    for (int k = n - 1; k >= 0; k--) {
      double t = b[k];
      b[k] = b[piv[k]];
      b[piv[k]] = t;
    }
  }
}

int orc_bruteforce(orc_net* n, const double* x, const double* u, const double* pd,
                   const double* qd, double sigma_f, double rho, const double* sigma_c,
                   const double* y, const double* s, const double* omega, double* H, double* J,
                   double* grad_u) {
  int nb = n->nb, nl = n->nl, nx = n->nx, nu = n->nu, m = n->m, nz = nx + nu;
  if (nb > 400) return ORC_EINVAL;
  bf_t B;
  memset(&B, 0, sizeof(B));
  B.n = n;
  B.pd = pd;
  B.qd = qd;
  B.Yr = (double*)xcalloc((size_t)nb * nb, sizeof(double));
  B.Yi = (double*)xcalloc((size_t)nb * nb, sizeof(double));
  double* arrs[8];
  for (int k = 0; k < 8; k++) arrs[k] = (double*)xcalloc((size_t)nl, sizeof(double));
  B.Yffr = arrs[0]; B.Yffi = arrs[1]; B.Yftr = arrs[2]; B.Yfti = arrs[3];
  B.Ytfr = arrs[4]; B.Ytfi = arrs[5]; B.Yttr = arrs[6]; B.Ytti = arrs[7];
  for (int l = 0; l < nl; l++) {
    int a = n->f[l], b = n->t[l];
    B.Yffr[l] = n->Gff[l]; B.Yffi[l] = n->Bff[l];
    B.Yftr[l] = n->Gft[l]; B.Yfti[l] = n->Bft[l];
    B.Ytfr[l] = n->Gtf[l]; B.Ytfi[l] = n->Btf[l];
    B.Yttr[l] = n->Gtt[l]; B.Ytti[l] = n->Btt[l];
    B.Yr[(size_t)a * nb + a] += n->Gff[l]; B.Yi[(size_t)a * nb + a] += n->Bff[l];
    B.Yr[(size_t)a * nb + b] += n->Gft[l]; B.Yi[(size_t)a * nb + b] += n->Bft[l];
    B.Yr[(size_t)b * nb + a] += n->Gtf[l]; B.Yi[(size_t)b * nb + a] += n->Btf[l];
    B.Yr[(size_t)b * nb + b] += n->Gtt[l]; B.Yi[(size_t)b * nb + b] += n->Btt[l];
  }
  hd* z = (hd*)xcalloc((size_t)nz, sizeof(hd));
  hd* g = (hd*)xcalloc((size_t)nx, sizeof(hd));
  hd* c = (hd*)xcalloc((size_t)m, sizeof(hd));
  double* zr = (double*)xcalloc((size_t)nz, sizeof(double));
  for (int i = 0; i < nx; i++) zr[i] = x[i];
  for (int j = 0; j < nu; j++) zr[nx + j] = u[j];
  /* base point values */
  for (int i = 0; i < nz; i++) z[i] = hd_c(zr[i]);
  hd cost;
  bf_eval(&B, z, g, c, &cost);
  double* c0 = (double*)xcalloc((size_t)m, sizeof(double));
  double* phid = (double*)xcalloc((size_t)m, sizeof(double));
  double* om = (double*)xcalloc((size_t)m, sizeof(double));
  for (int i = 0; i < m; i++) {
    c0[i] = c[i].a;
    phid[i] = y[i] * sigma_c[i] + rho * sigma_c[i] * sigma_c[i] * (c0[i] - s[i]);
    om[i] = omega ? omega[i] : rho * sigma_c[i] * sigma_c[i];
  }
  /* first derivatives (e1 only) */
  double* Jg = (double*)xcalloc((size_t)nx * nz, sizeof(double)); /* row-major nx x nz */
  double* Jcd = (double*)xcalloc((size_t)m * nz, sizeof(double));
  double* dF = (double*)xcalloc((size_t)nz, sizeof(double));
  for (int a = 0; a < nz; a++) {
    for (int i = 0; i < nz; i++) z[i] = hd_c(zr[i]);
    z[a].b = 1.0;
    bf_eval(&B, z, g, c, &cost);
    for (int i = 0; i < nx; i++) Jg[(size_t)i * nz + a] = g[i].b;
    for (int i = 0; i < m; i++) Jcd[(size_t)i * nz + a] = c[i].b;
    double d = sigma_f * cost.b;
    for (int i = 0; i < m; i++) d += phid[i] * c[i].b;
    dF[a] = d;
  }
  /* lambda: G_x^T lam = -d_x F */
  double* Gx = (double*)xcalloc((size_t)nx * nx, sizeof(double));
  int* piv = (int*)xcalloc((size_t)nx, sizeof(int));
  for (int i = 0; i < nx; i++)
    for (int j = 0; j < nx; j++) Gx[(size_t)i * nx + j] = Jg[(size_t)i * nz + j];
  int rc = dense_lu(nx, Gx, piv);
  double* lam = (double*)xcalloc((size_t)nx, sizeof(double));
  double* Smat = (double*)xcalloc((size_t)nx * nu, sizeof(double)); /* column-major nx x nu */
  double* K = (double*)xcalloc((size_t)nz * nz, sizeof(double));
  if (rc == ORC_OK) {
    for (int i = 0; i < nx; i++) lam[i] = -dF[i];
    dense_lu_solve(nx, Gx, piv, lam, 1);
    for (int j = 0; j < nu; j++) {
      double* col = Smat + (size_t)j * nx;
      for (int i = 0; i < nx; i++) col[i] = -Jg[(size_t)i * nz + nx + j];
      dense_lu_solve(nx, Gx, piv, col, 0);
    }
    if (grad_u)
      for (int j = 0; j < nu; j++) {
        double sacc = dF[nx + j];
        for (int i = 0; i < nx; i++) sacc += lam[i] * Jg[(size_t)i * nz + nx + j];
        grad_u[j] = sacc;
      }
    if (J) /* reduced Jacobian J = d_u c + d_x c S, m x nu column-major */
      for (int j = 0; j < nu; j++)
        for (int i = 0; i < m; i++) {
          double sacc = Jcd[(size_t)i * nz + nx + j];
          for (int k = 0; k < nx; k++) sacc += Jcd[(size_t)i * nz + k] * Smat[(size_t)j * nx + k];
          J[(size_t)j * m + i] = sacc;
        }
    /* second derivatives of l~ = sigma_f f + sum phid c + 1/2 sum om (c - c0)^2 + lam^T g */
    for (int a = 0; a < nz; a++)
      for (int b2 = a; b2 < nz; b2++) {
        for (int i = 0; i < nz; i++) z[i] = hd_c(zr[i]);
        z[a].b = 1.0;
        z[b2].c = 1.0;
        bf_eval(&B, z, g, c, &cost);
        double val = sigma_f * cost.d;
        for (int i = 0; i < m; i++) {
          hd dc = hd_sub(c[i], hd_c(c0[i]));
          val += phid[i] * c[i].d + 0.5 * om[i] * hd_mul(dc, dc).d;
        }
        for (int i = 0; i < nx; i++) val += lam[i] * g[i].d;
        K[(size_t)a * nz + b2] = val;
        K[(size_t)b2 * nz + a] = val;
      }
    /* H = K_uu + K_ux S + S^T K_xu + S^T K_xx S */
    if (H) {
      double* KS = (double*)xcalloc((size_t)nz * nu, sizeof(double)); /* K[:, x] S */
      for (int j = 0; j < nu; j++)
        for (int a = 0; a < nz; a++) {
          double sacc = 0.0;
          for (int k = 0; k < nx; k++) sacc += K[(size_t)a * nz + k] * Smat[(size_t)j * nx + k];
          KS[(size_t)j * nz + a] = sacc;
        }
      for (int j = 0; j < nu; j++)
        for (int i = 0; i < nu; i++) {
          double sacc = K[(size_t)(nx + i) * nz + nx + j] + KS[(size_t)j * nz + nx + i];
          for (int k = 0; k < nx; k++) {
            sacc += Smat[(size_t)i * nx + k] * K[(size_t)k * nz + nx + j];
            sacc += Smat[(size_t)i * nx + k] * KS[(size_t)j * nz + k];
          }
          H[(size_t)j * nu + i] = sacc;
        }
      free(KS);
    }
  }
  free(B.Yr);
  free(B.Yi);
  for (int k = 0; k < 8; k++) free(arrs[k]);
  free(z);
  free(g);
  free(c);
  free(zr);
  free(c0);
  free(phid);
  free(om);
  free(Jg);
  free(Jcd);
  free(dF);
  free(Gx);
  free(piv);
  free(lam);
  free(Smat);
  free(K);
  return rc;
}
